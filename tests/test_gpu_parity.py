"""GPU kernels against the FP64 oracle, element by element, through the C ABI.

Tolerances (relative 2-norm of the difference): 1e-12 for FP64 smoother
applications and operators, 1e-5 for FP32 (inputs rounded to FP32 on both
sides, oracle in FP64).  Sizes are small enough for the oracle to assemble
the global matrix and still span several blocks plus a ragged last block.
"""

import numpy as np
import pytest

from oracle import assembly, fe, multigrid, smoothers
from synthetic import normal_vector, uniform_vector

from gpu_helpers import TOL, as_prec, oracle_level, oracle_prolongation, rel_err, to_dev, to_host

pytestmark = pytest.mark.gpu

import paper_2405_19004_gb300 as vps  # noqa: E402

CASES = [(2, 1, 4), (2, 2, 4), (2, 3, 3), (2, 4, 3), (2, 5, 3), (2, 7, 2),
         (3, 1, 3), (3, 2, 3), (3, 3, 2), (3, 4, 2), (3, 5, 1), (3, 7, 1)]


def _poisson(d, k, l, prec, smoother=vps.VPS_MULTIPLICATIVE, damping=1.0):
    return vps.Poisson(d, k, l, precision=prec, smoother=smoother, damping=damping)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("d,k,l", CASES)
def test_colour_pass_matches_oracle(d, k, l, prec):
    lv, A, ps = oracle_level(d, k, l)
    P = _poisson(d, k, l, prec)
    x0 = as_prec(normal_vector(lv.N, 100 + d * 10 + k), prec)
    b = as_prec(normal_vector(lv.N, 200 + d * 10 + k), prec)
    for c in range(2 ** d):
        xg = to_dev(P, x0, l)
        P.vps_smooth_colour(l, c, to_dev(P, b, l), xg)
        got = to_host(P, xg, l)
        ref = smoothers.multiplicative(A, ps, x0, b, colours=[c])
        assert rel_err(got, ref) <= TOL[prec], (c, rel_err(got, ref))


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("d,k,l", [c for c in CASES if c[2] >= 2])
def test_multiplicative_step_matches_oracle(d, k, l, prec):
    lv, A, ps = oracle_level(d, k, l)
    P = _poisson(d, k, l, prec)
    x0 = as_prec(normal_vector(lv.N, 1 + k), prec)
    b = as_prec(normal_vector(lv.N, 2 + k), prec)
    xg = to_dev(P, x0, l)
    P.vps_smooth(l, to_dev(P, b, l), xg, 2)
    ref = smoothers.multiplicative(A, ps, smoothers.multiplicative(A, ps, x0, b), b)
    assert rel_err(to_host(P, xg, l), ref) <= TOL[prec]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("d,k,l", [(2, 2, 4), (2, 5, 3), (3, 2, 3), (3, 4, 2)])
def test_additive_step_matches_oracle(d, k, l, prec):
    lv, A, ps = oracle_level(d, k, l)
    P = _poisson(d, k, l, prec, vps.VPS_ADDITIVE, 0.7)
    x0 = as_prec(normal_vector(lv.N, 3), prec)
    b = as_prec(normal_vector(lv.N, 4), prec)
    xg = to_dev(P, x0, l)
    P.vps_smooth(l, to_dev(P, b, l), xg, 1)
    ref = smoothers.additive(A, ps, x0, b, 0.7)
    assert rel_err(to_host(P, xg, l), ref) <= TOL[prec]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("d,k,l", CASES)
def test_apply_matches_oracle(d, k, l, prec):
    lv, A, _ = oracle_level(d, k, l)
    P = _poisson(d, k, l, prec)
    x = as_prec(normal_vector(lv.N, 5), prec)
    y = P.empty_level(l)
    y.fill_(123.0)  # boundary entries must come back as 0
    P.vps_apply(l, to_dev(P, x, l), y)
    assert rel_err(to_host(P, y, l), A @ x) <= TOL[prec]
    n1 = lv.n1
    yy = y.double().cpu().numpy()
    px = P.layout(l)[1]
    assert yy[0] == 0.0 and yy[n1 - 1] == 0.0 and yy[px * (n1 - 1)] == 0.0


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("d,k,l", [(2, 1, 4), (2, 3, 3), (2, 7, 3), (3, 1, 3), (3, 2, 3), (3, 4, 2),
                                   (3, 6, 2)])
def test_transfers_match_oracle(d, k, l, prec):
    P = _poisson(d, k, l, prec)
    Pm = oracle_prolongation(d, k, l)
    nf, nc = Pm.shape
    xc = as_prec(normal_vector(nc, 6), prec)
    xf0 = as_prec(normal_vector(nf, 7), prec)
    xf = to_dev(P, xf0, l)
    P.vps_prolongate_add(l, to_dev(P, xc, l - 1), xf)
    assert rel_err(to_host(P, xf, l), xf0 + Pm @ xc) <= TOL[prec]
    rf = as_prec(normal_vector(nf, 8), prec)
    rc = P.empty_level(l - 1)
    rc.fill_(7.0)
    P.vps_restrict(l, to_dev(P, rf, l), rc)
    assert rel_err(to_host(P, rc, l - 1), Pm.T @ rf) <= TOL[prec]
    # boundary of the coarse output is zero
    n1c, pxc, _ = P.layout(l - 1)
    rr = rc.double().cpu().numpy()
    assert rr[n1c - 1] == 0.0 and rr[pxc * (n1c - 1) + 1] == 0.0


@pytest.mark.parametrize("coarse", [1, 0])
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("d,k,L,sm,om", [(2, 2, 4, 0, 1.0), (2, 3, 3, 1, 0.35), (3, 2, 3, 0, 1.0),
                                         (3, 3, 2, 1, 0.175), (2, 1, 5, 0, 1.0), (3, 1, 4, 0, 1.0)])
def test_vcycle_matches_oracle(d, k, L, sm, om, prec, coarse):
    P = _poisson(d, k, L, prec, sm, om)
    if coarse:
        P.vps_set_coarse_level(coarse)
    H = multigrid.Hierarchy(d, k, L, smoother="additive" if sm else "multiplicative", omega=om,
                            coarse_level=P.vps_get_coarse_level())
    b = as_prec(normal_vector(H.levels[L].N, 9), prec)
    x = P.empty_level(L)
    P.vps_vcycle(to_dev(P, b, L), x)
    tol = 1e-11 if prec == 0 else 1e-5
    assert rel_err(to_host(P, x, L), H.vcycle(L, b)) <= tol


@pytest.mark.parametrize("d,k,L", [(2, 3, 4), (3, 2, 3), (2, 7, 2), (3, 5, 2), (2, 7, 5), (2, 4, 6)])
def test_coarse_level_equal_to_finest_makes_the_vcycle_exact(d, k, L):
    """Global fast diagonalisation of a whole level is its exact inverse."""
    import scipy.sparse.linalg as spla
    lv, A, _ = oracle_level(d, k, L)
    P = _poisson(d, k, L, 0)
    P.vps_set_coarse_level(L)
    b = normal_vector(lv.N, 15)
    x = P.empty_level(L)
    P.vps_vcycle(to_dev(P, b, L), x)
    assert rel_err(to_host(P, x, L), spla.spsolve(A.tocsc(), b)) <= 1e-11


def test_default_coarse_level_rule():
    for d, k, L, want in [(3, 4, 5, 3), (2, 2, 4, 3), (3, 1, 6, 5), (3, 7, 4, 2), (2, 5, 1, 1)]:
        assert _poisson(d, k, L, 1).vps_get_coarse_level() == want


@pytest.mark.parametrize("d,k", [(2, 2), (3, 3), (2, 7)])
def test_level_one_vcycle_is_exact_solve(d, k):
    lv, A, _ = oracle_level(d, k, 1)
    P = _poisson(d, k, 1, 0)
    b = normal_vector(lv.N, 10)
    x = P.empty_level(1)
    P.vps_vcycle(to_dev(P, b, 1), x)
    import scipy.sparse.linalg as spla
    assert rel_err(to_host(P, x, 1), spla.spsolve(A.tocsc(), b)) <= 1e-12


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("d,k,L,sm,om", [(2, 2, 4, 0, 1.0), (3, 2, 3, 0, 1.0), (2, 3, 3, 1, 0.35),
                                         (3, 3, 3, 0, 1.0)])
def test_solve_matches_oracle(d, k, L, sm, om, prec):
    import torch
    P = _poisson(d, k, L, prec, sm, om)
    H = multigrid.Hierarchy(d, k, L, smoother="additive" if sm else "multiplicative", omega=om,
                            coarse_level=P.vps_get_coarse_level())
    A = H.A[L]
    b = uniform_vector(H.levels[L].N, 11)
    xo, ito, relo = multigrid.pcg(A, b, H.precondition, rtol=1e-10, max_it=100)
    bt = torch.as_tensor(b, device="cuda")
    xt = torch.zeros_like(bt)
    it, rel = P.vps_solve(bt, xt, 1e-10, 100)
    xg = xt.cpu().numpy()
    assert rel <= 1e-10
    assert np.linalg.norm(b - A @ xg) <= 1.01e-10 * np.linalg.norm(b)
    assert abs(it - ito) <= (0 if prec == 0 else 1)
    assert rel_err(xg, xo) <= 1e-8


def test_solve_host_matches_device_solve():
    import torch
    P = _poisson(3, 2, 3, 1)
    n = P.n_interior()
    b = torch.as_tensor(uniform_vector(n, 12)).pin_memory()
    x = torch.zeros(n, dtype=torch.float64).pin_memory()
    it, rel = P.vps_solve_host(b, x, 1e-10, 50)
    xd = torch.zeros(n, dtype=torch.float64, device="cuda")
    it2, rel2 = P.vps_solve(b.cuda(), xd, 1e-10, 50)
    assert it == it2 and rel <= 1e-10
    assert torch.equal(x, xd.cpu())


@pytest.mark.parametrize("d,k,L", [(2, 3, 3), (3, 2, 2)])
def test_rhs_assembly_matches_oracle(d, k, L):
    import torch
    from synthetic import sine_function, sine_modes
    coef, freq = sine_modes(d, 13)
    lv = fe.Level(d, k, L)
    ref = assembly.load_vector(lv, sine_function(coef, freq))
    P = _poisson(d, k, L, 0)
    b = torch.zeros(lv.N, dtype=torch.float64, device="cuda")
    P.vps_assemble_rhs_sines(coef, freq, b)
    assert rel_err(b.cpu().numpy(), ref) <= 1e-13


@pytest.mark.parametrize("d,k,L", [(2, 2, 3), (3, 1, 3)])
def test_l2_error_matches_oracle(d, k, L):
    import torch
    from synthetic import exact_sine_solution
    lv = fe.Level(d, k, L)
    x = normal_vector(lv.N, 14) * 0.01 + assembly.interpolate(lv, exact_sine_solution(d))
    ref = multigrid.l2_error(lv, x, exact_sine_solution(d))
    P = _poisson(d, k, L, 0)
    got = P.vps_l2_error_sine(torch.as_tensor(x, device="cuda"))
    assert abs(got - ref) <= 1e-12 * ref


def test_invalid_arguments_raise():
    P = _poisson(2, 2, 3, 0)
    x = P.empty_level(3)
    with pytest.raises(vps.VpsError) as e:
        P.vps_smooth(1, x, P.empty_level(1))  # level 1 has no smoother (single patch)
    assert e.value.code == vps.VPS_EINVAL
    with pytest.raises(vps.VpsError):
        P.vps_smooth_colour(3, 4, x, P.empty_level(3))
    with pytest.raises(vps.VpsError):
        P.vps_apply(4, x, P.empty_level(3))


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("d,k,l", [(2, 1, 4), (2, 2, 4), (2, 3, 4), (2, 6, 3), (2, 7, 2), (3, 1, 3), (3, 2, 3),
                                   (3, 3, 3), (3, 4, 2), (3, 5, 2), (3, 6, 2), (3, 7, 2)])
def test_every_smoother_variant_matches_oracle(d, k, l, prec):
    """Patches per block, warps per block and the fused / Boundary kernel
    (Section 3.2) are launch choices only: every variant gives the oracle's
    multiplicative step."""
    lv, A, ps = oracle_level(d, k, l)
    x0 = as_prec(normal_vector(lv.N, 31), prec)
    b = as_prec(normal_vector(lv.N, 32), prec)
    ref = smoothers.multiplicative(A, ps, x0, b)
    P = _poisson(d, k, l, prec)
    kinds = set()
    for v in range(vps.VPS_SMOOTH_VARIANTS):
        try:
            P.vps_set_smooth_variant(0, v)
        except vps.VpsError:
            continue  # does not fit in shared memory for this degree
        kinds.add(v // 3)
        xg = to_dev(P, x0, l)
        P.vps_smooth(l, to_dev(P, b, l), xg, 1)
        assert rel_err(to_host(P, xg, l), ref) <= TOL[prec], v
        # a colour pass at a time (the forward and the reverse order of a V-cycle)
        xg = to_dev(P, x0, l)
        bg = to_dev(P, b, l)
        for c in range(2 ** d):
            P.vps_smooth_colour(l, c, bg, xg)
        assert rel_err(to_host(P, xg, l), ref) <= TOL[prec], v
    want = {0, 1, 3, 4} | ({2} if k <= 3 else set())
    if k == 1 or (d == 2 and (k == 2 or (k == 3 and prec == vps.VPS_FP32))):
        want.add(5)  # one thread per patch
    assert kinds == want


def test_boundary_variants_are_multiplicative_only():
    P = _poisson(3, 2, 3, 1, 1, 0.175)
    for v in range(3, vps.VPS_SMOOTH_VARIANTS):
        with pytest.raises(vps.VpsError) as e:
            P.vps_set_smooth_variant(0, v)
        assert e.value.code == vps.VPS_EINVAL


def test_autotune_caches_and_keeps_parity(tmp_path):
    import torch
    cache = str(tmp_path / "tune.json")
    d, k, L = 3, 2, 4
    P = _poisson(d, k, L, 1)
    assert P.vps_autotune(cache) is False

    def choice(H):
        return ([H.vps_get_smooth_variant(l)[0] for l in range(1, L + 1)],
                [H.vps_get_operator_variant(l)[0] for l in range(1, L + 1)],
                H.vps_get_colour_schedule(), H.vps_get_coarse_level(), H.vps_get_coarse_solver())
    chosen = choice(P)
    assert [P.vps_get_operator_variant(l)[1] for l in range(1, L + 1)] == [2] * L  # 3D FP32 k <= 4
    Q = _poisson(d, k, L, 1)
    assert Q.vps_autotune(cache) is True
    assert choice(Q) == chosen
    import json
    entry = json.load(open(cache))
    assert len(entry) == 1
    (rec,) = entry.values()
    assert {"coarse", "variants", "ops", "schedule", "coarse_solver"} <= set(rec)
    H = multigrid.Hierarchy(d, k, L, coarse_level=Q.vps_get_coarse_level())
    b = uniform_vector(H.levels[L].N, 33)
    bt = torch.as_tensor(b, device="cuda")
    xt = torch.zeros_like(bt)
    it, rel = Q.vps_solve(bt, xt, 1e-10, 100)
    xo, ito, _ = multigrid.pcg(H.A[L], b, H.precondition, rtol=1e-10)
    assert rel <= 1e-10 and abs(it - ito) <= 1
    assert rel_err(xt.cpu().numpy(), xo) <= 1e-8


@pytest.mark.parametrize("op,schedule", [(1, 1), (0, 0), (1, 0), (1, 2), (0, 2)])
def test_operator_structure_and_colour_schedule_keep_parity(op, schedule):
    """Every tuning choice computes the same V-cycle: the alternative operator
    tile structure on every level and each colour schedule (ordinary,
    programmatic dependent launches, the dataflow sweep) against the
    oracle's V-cycle."""
    d, k, L = 3, 3, 4
    P = _poisson(d, k, L, 1)
    for l in range(2, L + 1):
        P.vps_set_operator_variant(l, op)
    P.vps_set_colour_schedule(schedule)
    H = multigrid.Hierarchy(d, k, L, coarse_level=P.vps_get_coarse_level())
    b = as_prec(uniform_vector(H.levels[L].N, 34), 1)
    x = P.empty_level(L)
    P.vps_vcycle(to_dev(P, b, L), x)
    assert rel_err(to_host(P, x, L), H.vcycle(L, b)) <= 1e-5


@pytest.mark.parametrize("prec", [0, 1])
def test_zero_right_hand_side_gives_zero_without_iterations(prec):
    """b = 0: x = 0 is the solution; the solve takes no iteration."""
    import torch
    P = _poisson(3, 2, 3, prec)
    b = torch.zeros(P.n_interior(), dtype=torch.float64, device="cuda")
    x = torch.full_like(b, 7.0)
    it, rel = P.vps_solve(b, x, 1e-10, 50)
    assert it == 0 and rel == 0.0
    assert torch.count_nonzero(x).item() == 0


@pytest.mark.parametrize("prec", [0, 1])
def test_non_finite_right_hand_side_is_a_breakdown(prec):
    """A NaN in b is reported as VPS_EBREAKDOWN, not as a result."""
    import torch
    P = _poisson(2, 2, 3, prec)
    b = torch.ones(P.n_interior(), dtype=torch.float64, device="cuda")
    b[5] = float("nan")
    x = torch.zeros_like(b)
    with pytest.raises(vps.VpsError) as e:
        P.vps_solve(b, x, 1e-10, 50)
    assert e.value.code == vps.VPS_EBREAKDOWN
