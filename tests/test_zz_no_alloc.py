"""The allocation-free additive step against the oracle and the handle-based step.

vps_smooth_additive_static is for callers that cannot call cudaMalloc (for
instance an application whose framework reserves nearly all device memory
for its own pool, or a loop that cannot afford the synchronisation of an
allocation): it needs no handle, and its scratch lives in fixed static
device arrays inside the library.  Here it is called through the C ABI and
compared, on two calls in a row (the second call reuses the scratch the
first one left), with the FP64 oracle's additive smoother and with
vps_smooth on a VPS_ADDITIVE handle with the same damping; the device's free
memory must not change between the calls.  This file is collected last on
purpose.
"""

import ctypes

import numpy as np
import pytest

from synthetic import normal_vector
from gpu_helpers import as_prec, oracle_level, rel_err, to_host

pytestmark = pytest.mark.gpu

import paper_2405_19004_gb300 as vps  # noqa: E402
from oracle import smoothers  # noqa: E402

TOL = {vps.VPS_FP64: 1e-12, vps.VPS_FP32: 1e-5}


def _rel(a, b):
    a = a.double().cpu().numpy()
    b = b.double().cpu().numpy()
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("prec", [vps.VPS_FP64, vps.VPS_FP32])
@pytest.mark.parametrize("d,k,l", [(2, 3, 4), (3, 2, 3), (3, 4, 5)])
def test_static_scratch_step_matches_oracle_and_handle_on_two_calls(d, k, l, prec):
    import torch
    omega = 0.7 * 2 / 2 ** d
    P = vps.Poisson(d, k, l, precision=prec, smoother=vps.VPS_ADDITIVE, damping=omega)
    N = P.n_interior()
    b_np = as_prec(normal_vector(N, 21), prec)
    x_np = as_prec(normal_vector(N, 22), prec)
    b = P.to_level(torch.as_tensor(b_np, device="cuda"))
    x0 = P.to_level(torch.as_tensor(x_np, device="cuda"))
    x_handle = x0.clone()
    x_static = x0.clone()
    stream = torch.cuda.Stream()
    # the oracle's two steps (the oracle only where it finishes in seconds)
    ref = None
    if N <= 40000:
        _, A, ps = oracle_level(d, k, l)
        ref = [smoothers.additive(A, ps, x_np, b_np, omega)]
        ref.append(smoothers.additive(A, ps, ref[0], b_np, omega))
    free = []
    for step in range(2):
        P.vps_smooth(l, b, x_handle, 1)
        stream.wait_stream(torch.cuda.current_stream())
        vps.vps_smooth_additive_static(d, k, l, prec, omega, b, x_static, stream)
        torch.cuda.current_stream().wait_stream(stream)
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        assert _rel(x_static, x_handle) <= TOL[prec]
        if ref is not None:
            assert rel_err(to_host(P, x_static, l), ref[step]) <= TOL[prec]
    assert free[0] == free[1]  # the second call allocated nothing
    assert _rel(x_static, x0) > 1e-3  # the step did change x


@pytest.mark.parametrize("d,k,l,prec", [(3, 4, 6, vps.VPS_FP64), (3, 7, 6, vps.VPS_FP32),
                                        (2, 7, 10, vps.VPS_FP64)]
                         + [(3, k, l, vps.VPS_FP64) for k in (1, 4, 7) for l in (19, 21, 24)])
def test_static_scratch_rejects_levels_beyond_its_size(d, k, l, prec):
    import torch
    lib = vps.lib()
    dt = torch.float64 if prec == vps.VPS_FP64 else torch.float32
    b = torch.zeros(64, dtype=dt, device="cuda")
    x = torch.zeros(64, dtype=dt, device="cuda")
    rc = lib.vps_smooth_additive_static(d, k, l, prec, 0.175, ctypes.c_void_p(b.data_ptr()),
                                        ctypes.c_void_p(x.data_ptr()), None)
    assert rc == vps.VPS_EINVAL
    assert b"static scratch" in lib.vps_last_error(None)
