"""The library's integer-instruction conversions between float and double
(used by the CG vector kernels in place of the FP64-pipe conversions)
against the GPU's own conversions, bit for bit, on patterns that cover every
class: zeros, subnormals, normals across and beyond the float range,
infinities, NaNs, ties of the rounding (both parities), carries of the
rounding into the exponent and up to infinity, and the edges of the exponent
ranges each fast path accepts."""
import numpy as np
import pytest
import torch

import paper_2405_19004_gb300 as vps

pytestmark = pytest.mark.gpu


def _patterns(seed=11, n=1 << 20):
    rng = np.random.default_rng(seed)
    parts = [rng.integers(0, 2**64, n, dtype=np.uint64)]  # every class, low 32 bits as floats too
    # doubles with biased exponents around and beyond the float range
    E = rng.integers(850, 1210, n, dtype=np.uint64)
    frac = rng.integers(0, 2**52, n, dtype=np.uint64)
    sign = rng.integers(0, 2, n, dtype=np.uint64) << np.uint64(63)
    parts.append(sign | (E << np.uint64(52)) | frac)
    # exact ties at the float rounding position, both parities of the kept bit
    tie = (frac & ~np.uint64(0x1FFFFFFF)) | np.uint64(1 << 28)
    parts.append(sign | (E << np.uint64(52)) | tie)
    parts.append(sign | (E << np.uint64(52)) | (tie ^ np.uint64(1 << 29)))
    # round-up carries into the exponent (all kept fraction bits set)
    parts.append(sign | (E << np.uint64(52)) | np.uint64(0xFFFFFFFFFFFFF))
    parts.append(sign | (E << np.uint64(52)) | (np.uint64(0xFFFFFF0000000) | (frac & np.uint64(0xFFFFFFF))))
    # the edges of the accepted exponent ranges, every fraction class
    edges = np.array([0, 1, 895, 896, 897, 898, 948, 949, 950, 951, 1149, 1150, 1151, 1152, 2046, 2047],
                     dtype=np.uint64)
    m = 4096
    Ee = edges[rng.integers(0, len(edges), m)]
    parts.append(rng.integers(0, 2, m, dtype=np.uint64) << np.uint64(63) | (Ee << np.uint64(52))
                 | rng.integers(0, 2**52, m, dtype=np.uint64))
    # floats of every class in the low 32 bits
    fe = rng.integers(0, 256, n, dtype=np.uint64)
    parts.append((rng.integers(0, 2, n, dtype=np.uint64) << np.uint64(31)) | (fe << np.uint64(23))
                 | rng.integers(0, 2**23, n, dtype=np.uint64))
    special = [0, 1 << 63, 0x7FF0000000000000, 0xFFF0000000000000, 0x7FF8000000000000,
               0x0000000000000001, 0x000FFFFFFFFFFFFF, 0x3FF0000000000000, 0x47EFFFFFE0000000,
               0x47EFFFFFF0000000, 0x47EFFFFFEFFFFFFF, 0x3810000000000000, 0x380FFFFFFFFFFFFF,
               0x0000000080000000, 0x000000007F800000, 0x000000007FC00000, 0x0000000000000001,
               0x00000000807FFFFF]
    parts.append(np.array(special, dtype=np.uint64))
    allp = np.concatenate(parts)
    return torch.from_numpy(allp.view(np.int64)).cuda()


def test_conversions_match_the_hardware():
    pat = _patterns()
    s = torch.cuda.current_stream()
    bad = vps.vps_check_fp_conversions(pat, s)
    assert bad == [0, 0, 0], bad


def test_conversions_empty_and_errors():
    s = torch.cuda.current_stream()
    assert vps.vps_check_fp_conversions(torch.zeros(0, dtype=torch.int64, device="cuda"), s) == [0, 0, 0]
    L = vps.lib()
    import ctypes
    out = (ctypes.c_int64 * 3)()
    assert L.vps_check_fp_conversions(None, 4, out, None) == vps.VPS_EINVAL
