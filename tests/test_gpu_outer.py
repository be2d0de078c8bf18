"""The outer CG operator: FP64 and double-float evaluation of A p (Section 4.2).

The double-float operator evaluates the same sum-factorised product with each
value held as a pair of floats; its results are compared with the oracle's
assembled matrix at the FP64 bar (1e-12 relative), on random vectors (no
cancellation) and on a smooth vector (the terms cancel to O(h^2) of their
size), where the bound is stated against max (|A| |x|), the scale of the
floating-point error of any evaluation of the sum.  The mixed-precision
solve must reach the same tolerance on the true FP64 residual whichever
outer operator it uses.
"""

import numpy as np
import pytest

from synthetic import normal_vector, uniform_vector

from gpu_helpers import oracle_level

pytestmark = pytest.mark.gpu

import paper_2405_19004_gb300 as vps  # noqa: E402

CASES = [(2, 1, 4), (2, 3, 3), (2, 7, 2), (3, 1, 3), (3, 2, 3), (3, 4, 2), (3, 5, 2), (3, 7, 1)]


def _pack64(P, x, xl):
    """Pack a compact FP64 vector into the finest level's layout (padding 0)."""
    import torch
    d, n1 = P.dim, P.layout(P.level)[0]
    px = P.layout(P.level)[1]
    ni = n1 - 2
    v = torch.as_tensor(x, device="cuda").reshape((ni,) * d)
    if d == 3:
        full = xl.view(n1, n1, px)
        full[1:n1 - 1, 1:n1 - 1, 1:n1 - 1] = v
    else:
        full = xl.view(n1, px)
        full[1:n1 - 1, 1:n1 - 1] = v


def _unpack64(P, y):
    d, (n1, px, _) = P.dim, P.layout(P.level)
    if d == 3:
        full = y.view(n1, n1, px)
        inner = full[1:n1 - 1, 1:n1 - 1, 1:n1 - 1]
    else:
        full = y.view(n1, px)
        inner = full[1:n1 - 1, 1:n1 - 1]
    return inner.reshape(-1).cpu().numpy(), full


@pytest.mark.parametrize("mode", [vps.VPS_OUTER_FP64, vps.VPS_OUTER_DOUBLE_FLOAT], ids=["fp64", "df"])
@pytest.mark.parametrize("prec", [vps.VPS_FP64, vps.VPS_FP32], ids=["h64", "h32"])
@pytest.mark.parametrize("d,k,l", CASES)
def test_outer_operator_matches_oracle(d, k, l, prec, mode):
    import torch
    lv, A, _ = oracle_level(d, k, l)
    P = vps.Poisson(d, k, l, precision=prec)
    P.vps_set_outer_operator(mode)
    assert P.vps_get_outer_operator() == mode
    absA = abs(A)
    for x in (normal_vector(lv.N, 61), np.sin(np.pi * np.linspace(0.05, 0.95, lv.N)) + 1.0):
        xl = P.empty_level(l, dtype=torch.float64)
        _pack64(P, x, xl)
        y = xl.clone().fill_(123.0)
        P.vps_apply_outer(xl, y)
        got, full = _unpack64(P, y)
        ref = A @ x
        scale = (absA @ np.abs(x)).max()
        assert np.abs(got - ref).max() <= 1e-12 * scale
        # boundary nodes come back 0 (padding columns beyond n1 are not written)
        n1 = P.layout(l)[0]
        box = full[..., :n1].cpu().numpy()
        inner = np.zeros(box.shape, dtype=bool)
        inner[(slice(1, n1 - 1),) * d] = True
        assert np.all(box[~inner] == 0.0)
    # random vectors: the relative 2-norm error at the FP64 bar
    x = normal_vector(lv.N, 62)
    xl = P.empty_level(l, dtype=torch.float64)
    _pack64(P, x, xl)
    y = xl.clone()
    P.vps_apply_outer(xl, y)
    got, _ = _unpack64(P, y)
    ref = A @ x
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)


def test_fp32_handle_defaults_to_double_float():
    assert vps.Poisson(3, 2, 2, precision=vps.VPS_FP32).vps_get_outer_operator() == \
        vps.VPS_OUTER_DOUBLE_FLOAT
    assert vps.Poisson(3, 2, 2, precision=vps.VPS_FP64).vps_get_outer_operator() == vps.VPS_OUTER_FP64


def test_outer_operator_rejects_unknown_mode():
    P = vps.Poisson(2, 2, 2, precision=vps.VPS_FP32)
    with pytest.raises(vps.VpsError) as e:
        P.vps_set_outer_operator(2)
    assert e.value.code == vps.VPS_EINVAL
    assert P.vps_get_outer_operator() == vps.VPS_OUTER_DOUBLE_FLOAT


@pytest.mark.parametrize("rtol", [1e-10, 1e-12])
@pytest.mark.parametrize("d,k,L", [(3, 3, 3), (2, 4, 4), (3, 2, 4)])
def test_mixed_solve_with_either_outer_operator(d, k, L, rtol):
    import torch
    lv, A, _ = oracle_level(d, k, L)
    b = uniform_vector(lv.N, 63)
    sols, its = {}, {}
    for mode in (vps.VPS_OUTER_FP64, vps.VPS_OUTER_DOUBLE_FLOAT):
        P = vps.Poisson(d, k, L, precision=vps.VPS_FP32)
        P.vps_set_outer_operator(mode)
        bt = torch.as_tensor(b, device="cuda")
        xt = torch.zeros_like(bt)
        it, rel = P.vps_solve(bt, xt, rtol, 100)
        x = xt.cpu().numpy()
        true_rel = np.linalg.norm(b - A @ x) / np.linalg.norm(b)
        assert rel <= rtol
        # the reported residual is an FP64 residual: it agrees with the oracle's
        assert true_rel <= 1.02 * rtol, (mode, true_rel)
        sols[mode], its[mode] = x, it
    assert abs(its[0] - its[1]) <= 2
    dx = np.linalg.norm(sols[0] - sols[1]) / np.linalg.norm(sols[0])
    assert dx <= 100 * rtol


def _gamma(k):
    return (6 * k + 6) * 2.0 ** -53


@pytest.mark.parametrize("prec,mode", [(vps.VPS_FP32, vps.VPS_OUTER_DOUBLE_FLOAT),
                                       (vps.VPS_FP32, vps.VPS_OUTER_FP64),
                                       (vps.VPS_FP64, vps.VPS_OUTER_FP64)])
@pytest.mark.parametrize("d,k,L", [(2, 2, 7), (2, 5, 5)])
def test_unattainable_rtol_ends_at_the_rounding_bound(d, k, L, prec, mode):
    """2D meshes with a smooth right-hand side: the terms of A x cancel by
    about k^2 h^-2, so rtol = 1e-15 cannot be shown in FP64.  The solve ends
    (VPS_OK) once the FP64 residual is within the rounding bound of its own
    evaluation, checked here against the oracle's assembled matrix."""
    import torch
    from synthetic import sine_modes
    lv, A, _ = oracle_level(d, k, L)
    P = vps.Poisson(d, k, L, precision=prec)
    P.vps_set_outer_operator(mode)
    coef, freq = sine_modes(d, 64)
    b = torch.zeros(lv.N, dtype=torch.float64, device="cuda")
    P.vps_assemble_rhs_sines(coef, freq, b)
    x = torch.zeros_like(b)
    it, rel = P.vps_solve(b, x, 1e-15, 200)
    restarts, at_bound = P.vps_get_solve_info()
    assert at_bound == 1 and it < 60
    bh, xh = b.cpu().numpy(), x.cpu().numpy()
    r = np.linalg.norm(bh - A @ xh)
    U = np.linalg.norm(abs(A) @ np.abs(xh))
    assert r <= 4 * _gamma(k) * U
    assert abs(rel - r / np.linalg.norm(bh)) <= 0.5 * rel + 4 * _gamma(k) * U / np.linalg.norm(bh)


def test_attainable_rtol_does_not_use_the_rounding_bound():
    import torch
    d, k, L = 3, 4, 3
    lv, A, _ = oracle_level(d, k, L)
    P = vps.Poisson(d, k, L, precision=vps.VPS_FP32)
    b = torch.as_tensor(uniform_vector(lv.N, 65), device="cuda")
    x = torch.zeros_like(b)
    it, rel = P.vps_solve(b, x, 1e-10, 100)
    assert P.vps_get_solve_info() == (0, 0)
    true_rel = np.linalg.norm(b.cpu().numpy() - A @ x.cpu().numpy()) / np.linalg.norm(b.cpu().numpy())
    assert true_rel <= 1.02e-10 and abs(true_rel - rel) <= 1e-3 * rel


def test_server_requests_with_unattainable_rtol_complete():
    from synthetic import sine_modes
    srv = vps.Server(4 << 30, max_active=3, precision=vps.VPS_FP32, rtol=1e-15, max_it=200)
    ids = []
    for i, (d, k, L) in enumerate([(2, 2, 7), (2, 5, 5), (3, 2, 3)]):
        coef, freq = sine_modes(d, 70 + i)
        ids.append(srv.submit(d, k, L, coef, freq)[0])
    srv.wait(0, 300)
    info = [srv.query(r) for r in ids]
    srv.close()
    for q in info:
        assert q["state"] == vps.VPS_REQ_DONE, q


@pytest.mark.parametrize("prec", [vps.VPS_FP32, vps.VPS_FP64], ids=["h32", "h64"])
@pytest.mark.parametrize("rtol", [1e-10, 1e-13])
def test_device_loop_equals_host_loop(prec, rtol):
    """With graphs the CG iterations after the first run on the device (a
    conditional while-node); without, every iteration returns to the host.
    Same kernels in the same order: bit-identical solutions and counts (also
    through the restarts an unattainable rtol forces)."""
    import torch
    d, k, L = 2, 2, 6
    out = []
    for graphs in (True, False):
        P = vps.Poisson(d, k, L, precision=prec)
        P.vps_set_graphs(graphs)
        b = torch.as_tensor(uniform_vector(P.n_interior(), 66), device="cuda")
        x = torch.zeros_like(b)
        it, rel = P.vps_solve(b, x, rtol, 200)
        out.append((it, rel, P.vps_get_solve_info(), x.cpu()))
    assert out[0][:3] == out[1][:3]
    assert torch.equal(out[0][3], out[1][3])
