"""Continuous-batching server: correctness, isolation between requests, admission.

A request's result must not depend on what else runs: it is compared bit for
bit between a run alone and a run in a mix of concurrent requests, whose
V-cycles share batched launches with the other requests of their cohort
(same dimension and degree).
"""

import numpy as np
import pytest

from oracle import assembly, fe
from synthetic import sine_function, sine_modes

pytestmark = pytest.mark.gpu

import paper_2405_19004_gb300 as vps  # noqa: E402

SHAPES = [(2, 2, 4), (3, 2, 3), (2, 5, 3), (3, 3, 3), (2, 3, 5), (3, 4, 3), (2, 2, 4), (3, 2, 3),
          (2, 6, 2), (3, 1, 4), (2, 4, 4), (3, 5, 2)]
GB = 1 << 30


def _requests():
    out = []
    for i, (d, k, L) in enumerate(SHAPES):
        coef, freq = sine_modes(d, 100 + i)
        out.append((d, k, L, coef, freq))
    return out


def _run(requests, max_active, alone):
    srv = vps.Server(8 * GB, max_active=max_active, precision=vps.VPS_FP32)
    ids, xs = [], []
    for (d, k, L, coef, freq) in requests:
        rid, x = srv.submit(d, k, L, coef, freq)
        ids.append(rid)
        xs.append(x)
        if alone:
            srv.wait(rid, 120)
    srv.wait(0, 300)
    info = [srv.query(r) for r in ids]
    srv.close()
    return xs, info


def test_results_alone_and_in_a_mix_are_identical():
    reqs = _requests()
    x_alone, info_alone = _run(reqs, 1, alone=True)
    x_mix, info_mix = _run(reqs, 6, alone=False)
    for a, b, ia, ib in zip(x_alone, x_mix, info_alone, info_mix):
        assert ia["state"] == vps.VPS_REQ_DONE and ib["state"] == vps.VPS_REQ_DONE
        assert ia["iters"] == ib["iters"]
        assert np.array_equal(a, b)
        assert ib["latency_s"] >= ib["queue_s"] >= 0.0


def test_served_solutions_satisfy_the_oracle_system():
    srv = vps.Server(4 * GB, max_active=3, precision=vps.VPS_FP32)
    out = []
    for (d, k, L, coef, freq) in _requests()[:5]:
        rid, x = srv.submit(d, k, L, coef, freq)
        out.append((rid, x, d, k, L, coef, freq))
    srv.wait(0, 300)
    for rid, x, d, k, L, coef, freq in out:
        info = srv.query(rid)
        assert info["state"] == vps.VPS_REQ_DONE and info["rel_res"] <= 1e-10
        lv = fe.Level(d, k, L)
        A = assembly.stiffness(lv)
        b = assembly.load_vector(lv, sine_function(coef, freq))
        assert np.linalg.norm(b - A @ x) <= 1.05e-10 * np.linalg.norm(b)
    srv.close()


def test_server_matches_a_handle_solve():
    import torch
    d, k, L, coef, freq = _requests()[3]
    srv = vps.Server(GB, max_active=1)
    rid, x = srv.submit(d, k, L, coef, freq)
    srv.wait(rid, 120)
    P = vps.Poisson(d, k, L, precision=vps.VPS_FP32)
    b = torch.zeros(P.n_interior(), dtype=torch.float64, device="cuda")
    P.vps_assemble_rhs_sines(coef, freq, b)
    xt = torch.zeros_like(b)
    P.vps_solve(b, xt, 1e-10, 100)
    assert np.array_equal(x, xt.cpu().numpy())
    srv.close()


def test_tight_budget_evicts_idle_hierarchies_and_still_serves_everything():
    # each hierarchy fits (about 85 MB and 30 MB) but not both at once
    srv = vps.Server(100 << 20, max_active=2, precision=vps.VPS_FP32)
    reqs = [(3, 3, 5), (3, 4, 4), (3, 3, 5), (3, 4, 4), (3, 3, 5)]
    ids = []
    for i, (d, k, L) in enumerate(reqs):
        coef, freq = sine_modes(d, 200 + i)
        ids.append(srv.submit(d, k, L, coef, freq)[0])
    srv.wait(0, 300)
    for rid in ids:
        info = srv.query(rid)
        assert info["state"] == vps.VPS_REQ_DONE, (info, srv.last_error())
    srv.close()


def test_request_larger_than_the_budget_fails_cleanly():
    srv = vps.Server(1 << 20, max_active=2)
    coef, freq = sine_modes(3, 7)
    rid, _ = srv.submit(3, 4, 4, coef, freq)
    srv.wait(rid, 60)
    info = srv.query(rid)
    assert info["state"] == vps.VPS_REQ_FAILED and info["status"] == vps.VPS_ENOMEM
    srv.close()


def test_wait_times_out_on_the_host():
    srv = vps.Server(GB, max_active=1)
    coef, freq = sine_modes(3, 8)
    rid, _ = srv.submit(3, 4, 4, coef, freq)
    with pytest.raises(vps.VpsError) as e:
        srv.wait(rid, 1e-6)
    assert e.value.code == vps.VPS_ETIMEOUT
    srv.wait(rid, 120)
    assert srv.query(rid)["state"] == vps.VPS_REQ_DONE
    srv.close()


def test_requests_of_one_cohort_share_batched_launches():
    """Four 3D Q2 requests of three levels: a first round builds their
    hierarchies; in the second round all four have a resident slot, are
    admitted together and run as one cohort, so batched launches process
    tiles of several requests.  Each result still equals the request's result
    alone."""
    reqs = [(3, 2, 3), (3, 2, 4), (3, 2, 3), (3, 2, 2)]
    coefs = [sine_modes(3, 300 + i) for i in range(len(reqs))]
    srv = vps.Server(4 * GB, max_active=8, precision=vps.VPS_FP32)
    for i, (d, k, L) in enumerate(reqs):
        srv.submit(d, k, L, *coefs[i])
    srv.wait(0, 300)
    before = srv.batch_stats()
    xs = [srv.submit(d, k, L, *coefs[i])[1] for i, (d, k, L) in enumerate(reqs)]
    srv.wait(0, 300)
    st = srv.batch_stats()
    srv.close()
    assert st["max_requests_per_launch"] >= 2 and st["max_requests_per_tick"] >= 2, (before, st)
    assert st["batched_launches"] > before["batched_launches"] and st["ticks"] > before["ticks"]
    for i, (d, k, L) in enumerate(reqs):
        alone = vps.Server(GB, max_active=1, precision=vps.VPS_FP32)
        rid, x = alone.submit(d, k, L, *coefs[i])
        alone.wait(rid, 120)
        assert alone.query(rid)["state"] == vps.VPS_REQ_DONE
        alone.close()
        assert np.array_equal(x, xs[i])


def test_submit_rejects_levels_beyond_the_size_limit():
    """The size check runs before any size is computed from the level, so
    levels whose element count would overflow an integer are rejected too."""
    srv = vps.Server(GB, max_active=1)
    coef, freq = sine_modes(3, 9)
    for L in (11, 19, 24):
        with pytest.raises(vps.VpsError) as e:
            srv.submit(3, 7, L, coef, freq)
        assert e.value.code == vps.VPS_EINVAL
    srv.close()
