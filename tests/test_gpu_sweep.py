"""The dataflow sweep of the multiplicative smoother: a whole smoothing step
as one launch of one block per tile of every colour, each tile waiting for
the overlapping patches of the earlier colours.

Checked against the oracle's multiplicative smoother (Algorithm 3, colours
in order) at the parity tolerances, against the colour-by-colour launches
bit for bit (every variant with a sweep kernel, both precisions, levels from
a handful of tiles per colour up to the 3D Q4 workload's finest level), in
V-cycles and CG solves (CUDA graphs, several sweeps in a row, both colour
orders), and with the bounded dependency wait made to expire from the host
(tiles skipped by the fault-injection hook): the wait reports VPS_ETIMEOUT
and the next sweep is correct again.
"""

import pytest

from oracle import multigrid, smoothers
from synthetic import normal_vector, uniform_vector

from gpu_helpers import TOL, as_prec, oracle_level, rel_err, to_dev, to_host

pytestmark = pytest.mark.gpu

import paper_2405_19004_gb300 as vps  # noqa: E402

PLAIN, PDL, SWEEP = vps.VPS_SCHEDULE_PLAIN, vps.VPS_SCHEDULE_PDL, vps.VPS_SCHEDULE_SWEEP


def _smooth(P, level, x0, b, schedule, steps=2):
    P.vps_set_colour_schedule(schedule)
    xg = to_dev(P, x0, level)
    P.vps_smooth(level, to_dev(P, b, level), xg, steps)
    P.vps_check_waits()
    return xg


def _variants(P, level):
    """The smoother variants of `level` that have a sweep kernel (0-5, 9-14) and fit."""
    out = []
    for v in list(range(6)) + list(range(9, 15)):
        try:
            P.vps_set_smooth_variant(level, v)
        except vps.VpsError:
            continue
        out.append(v)
    return out


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("d,k,l", [(2, 1, 4), (2, 3, 3), (2, 5, 3), (2, 7, 2),
                                   (3, 1, 3), (3, 2, 3), (3, 4, 2), (3, 6, 2)])
def test_sweep_step_matches_oracle(d, k, l, prec):
    lv, A, ps = oracle_level(d, k, l)
    P = vps.Poisson(d, k, l, precision=prec)
    x0 = as_prec(normal_vector(lv.N, 41 + k), prec)
    b = as_prec(normal_vector(lv.N, 42 + k), prec)
    ref = smoothers.multiplicative(A, ps, smoothers.multiplicative(A, ps, x0, b), b)
    for v in _variants(P, l):
        xg = _smooth(P, l, x0, b, SWEEP)
        assert rel_err(to_host(P, xg, l), ref) <= TOL[prec], v


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("d,k,l", [(2, 1, 6), (2, 2, 5), (2, 4, 4), (2, 6, 4), (2, 7, 3),
                                   (3, 1, 5), (3, 2, 4), (3, 3, 4), (3, 4, 3), (3, 5, 3),
                                   (3, 6, 2), (3, 7, 2)])
def test_sweep_equals_colour_passes_bit_for_bit(d, k, l, prec):
    import torch
    P = vps.Poisson(d, k, l, precision=prec)
    x0 = as_prec(normal_vector(_compact_size(P, l), 43), prec)
    b = as_prec(normal_vector(_compact_size(P, l), 44), prec)
    for v in _variants(P, l):
        ref = _smooth(P, l, x0, b, PLAIN)
        got = _smooth(P, l, x0, b, SWEEP)
        assert torch.equal(got, ref), (v, (got - ref).abs().max().item())


def _compact_size(P, level):
    n1 = P.layout(level)[0]
    return (n1 - 2) ** P.dim


@pytest.mark.parametrize("prec", [1, 0])
def test_sweep_at_the_workload_size_equals_colour_passes(prec):
    """3D Q4 on 2^5 cells (the bench's finest level, 2,048,383 DoFs): many
    tiles per colour, blocks far beyond one wave."""
    import torch
    P = vps.Poisson(3, 4, 5, precision=prec)
    n = _compact_size(P, 5)
    x0 = as_prec(normal_vector(n, 45), prec)
    b = as_prec(normal_vector(n, 46), prec)
    for v in _variants(P, 5):
        ref = _smooth(P, 5, x0, b, PDL, steps=3)
        got = _smooth(P, 5, x0, b, SWEEP, steps=3)
        assert torch.equal(got, ref), v


@pytest.mark.parametrize("d,k,L,pre,post", [(3, 4, 4, 1, 1), (3, 2, 4, 2, 2), (2, 3, 5, 1, 1)])
def test_sweep_vcycle_and_solve_equal_colour_passes(d, k, L, pre, post):
    """V-cycles (forward pre-smoothing, backward post-smoothing, several sweeps
    in a row) and CG solves through CUDA graphs: the same bits with either
    schedule, and the oracle's V-cycle."""
    import torch
    res = {}
    for schedule in (PDL, SWEEP):
        P = vps.Poisson(d, k, L, precision=vps.VPS_FP32, n_pre=pre, n_post=post)
        P.vps_set_colour_schedule(schedule)
        n = P.n_interior()
        b = torch.as_tensor(uniform_vector(n, 47), device="cuda")
        x = torch.zeros_like(b)
        it, rel = P.vps_solve(b, x, 1e-10, 100)
        bl = to_dev(P, as_prec(uniform_vector(n, 48), 1), L)
        xl = P.empty_level(L)
        P.vps_vcycle(bl, xl)
        P.vps_check_waits()
        res[schedule] = (it, x, xl, P.vps_get_coarse_level())
    assert res[PDL][0] == res[SWEEP][0]
    assert torch.equal(res[PDL][1], res[SWEEP][1])
    assert torch.equal(res[PDL][2], res[SWEEP][2])
    if pre == 1 and post == 1:
        H = multigrid.Hierarchy(d, k, L, coarse_level=res[SWEEP][3])
        P = vps.Poisson(d, k, L, precision=vps.VPS_FP32)
        got = to_host(P, res[SWEEP][2], L)
        assert rel_err(got, H.vcycle(L, as_prec(uniform_vector(H.levels[L].N, 48), 1))) <= 1e-5


def test_expired_dependency_wait_is_reported_and_the_next_sweep_is_correct():
    """Tiles of the first colour skipped from the host: the tiles of later
    colours that overlap them wait until the poll limit (about a second),
    the sweep finishes, VPS_ETIMEOUT is reported, and the context, the
    counters and the flags serve the next sweep correctly."""
    import torch
    d, k, l = 3, 2, 4
    P = vps.Poisson(d, k, l, precision=vps.VPS_FP32)
    n = _compact_size(P, l)
    x0 = as_prec(normal_vector(n, 49), 1)
    b = as_prec(normal_vector(n, 50), 1)
    ref = _smooth(P, l, x0, b, PLAIN, steps=1)
    P.vps_set_colour_schedule(SWEEP)
    P.vps_skip_sweep_tiles(l, 4)
    xg = to_dev(P, x0, l)
    P.vps_smooth(l, to_dev(P, b, l), xg, 1)
    with pytest.raises(vps.VpsError) as e:
        P.vps_check_waits()
    assert e.value.code == vps.VPS_ETIMEOUT
    P.vps_check_waits()  # the record was cleared
    got = _smooth(P, l, x0, b, SWEEP, steps=1)
    assert torch.equal(got, ref)


def test_schedule_argument_checked():
    P = vps.Poisson(2, 2, 3)
    with pytest.raises(vps.VpsError):
        P.vps_set_colour_schedule(3)
    with pytest.raises(vps.VpsError):
        P.vps_skip_sweep_tiles(4, 0)
    assert P.vps_get_colour_schedule() == PDL
