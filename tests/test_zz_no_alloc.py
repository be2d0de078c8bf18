"""The allocation-free additive step against the handle-based one.

vps_smooth_additive_static is for callers that cannot call cudaMalloc (for
instance an application whose framework reserves nearly all device memory
for its own pool, or a loop that cannot afford the synchronisation of an
allocation): it needs no handle, and its scratch lives in a fixed static
device array inside the library.  Here it is called through the C ABI and
compared with vps_smooth on a VPS_ADDITIVE handle with the same damping, on
two calls in a row (the second call reuses the scratch the first one left).
This file is collected last on purpose.
"""

import numpy as np
import pytest

from synthetic import normal_vector

pytestmark = pytest.mark.gpu

import paper_2405_19004_gb300 as vps  # noqa: E402

TOL = {vps.VPS_FP64: 1e-12, vps.VPS_FP32: 1e-5}


def _rel(a, b):
    a = a.double().cpu().numpy()
    b = b.double().cpu().numpy()
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("prec", [vps.VPS_FP64, vps.VPS_FP32])
@pytest.mark.parametrize("d,k,l", [(2, 3, 4), (3, 2, 3), (3, 4, 5)])
def test_static_scratch_step_matches_handle_step_on_two_calls(d, k, l, prec):
    import torch
    omega = 0.7 * 2 / 2 ** d
    P = vps.Poisson(d, k, l, precision=prec, smoother=vps.VPS_ADDITIVE, damping=omega)
    N = P.n_interior()
    b = P.to_level(torch.as_tensor(normal_vector(N, 21), device="cuda"))
    x0 = P.to_level(torch.as_tensor(normal_vector(N, 22), device="cuda"))
    x_handle = x0.clone()
    x_static = x0.clone()
    stream = torch.cuda.Stream()
    for _ in range(2):
        P.vps_smooth(l, b, x_handle, 1)
        stream.wait_stream(torch.cuda.current_stream())
        vps.vps_smooth_additive_static(d, k, l, prec, omega, b, x_static, stream)
        torch.cuda.current_stream().wait_stream(stream)
        torch.cuda.synchronize()
        assert _rel(x_static, x_handle) <= TOL[prec]
    assert _rel(x_static, x0) > 1e-3  # the step did change x


def test_static_scratch_rejects_levels_beyond_its_size():
    import ctypes
    lib = vps.lib()
    dummy = ctypes.c_void_p(16)
    rc = lib.vps_smooth_additive_static(3, 4, 6, vps.VPS_FP64, 0.175, dummy, ctypes.c_void_p(32),
                                        None)
    assert rc == vps.VPS_EINVAL
    assert b"static scratch" in lib.vps_last_error(None)
