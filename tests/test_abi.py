"""The C-ABI library builds, loads and exports every symbol include/*.h declares.

No compute calls: these run without a GPU.  Argument validation happens
before any CUDA call, so invalid vps_create arguments are checked here too.
"""

import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(vps_[a-z0-9_]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2405_19004_gb300 as vps
    return vps.lib()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert {"vps_create", "vps_smooth", "vps_vcycle", "vps_solve", "vps_apply"} <= names
    for n in sorted(names):
        assert hasattr(lib, n), n


def test_binding_signatures_cover_the_header(lib):
    import paper_2405_19004_gb300 as vps
    assert _declared() <= set(vps.SIGNATURES)


@pytest.mark.parametrize("args,needle", [
    ((4, 2, 3, 0, 0, 1.0, 1, 1), "dim"),
    ((2, 0, 3, 0, 0, 1.0, 1, 1), "degree"),
    ((2, 8, 3, 0, 0, 1.0, 1, 1), "degree"),
    ((2, 2, 0, 0, 0, 1.0, 1, 1), "level"),
    ((2, 2, 3, 7, 0, 1.0, 1, 1), "precision"),
    ((2, 2, 3, 0, 5, 1.0, 1, 1), "smoother"),
    ((2, 2, 3, 0, 0, 0.0, 1, 1), "damping"),
    ((2, 2, 3, 0, 0, float("nan"), 1, 1), "damping"),
    ((2, 2, 3, 0, 0, 1.0, -1, 1), "n_pre"),
    ((3, 7, 11, 0, 0, 1.0, 1, 1), "too large"),
])
def test_create_rejects_invalid_arguments_without_touching_cuda(lib, args, needle):
    h = ctypes.c_void_p()
    rc = lib.vps_create(*args, None, ctypes.byref(h))
    assert rc == -1 and not h.value
    assert needle in lib.vps_last_error(None).decode()


def test_status_strings_and_null_handles(lib):
    assert lib.vps_status_string(0) == b"VPS_OK"
    assert lib.vps_status_string(-5) == b"VPS_EBREAKDOWN"
    assert lib.vps_destroy(None) == 0
    assert lib.vps_smooth(None, 2, None, None, 1) == -1
    assert lib.vps_sizes(None, None, None, None) == -1


def test_no_cpu_fallback_in_the_package():
    """The product package never imports the oracle."""
    pkg = os.path.join(ROOT, "paper_2405_19004_gb300")
    for f in glob.glob(os.path.join(pkg, "**", "*.py"), recursive=True):
        src = open(f).read()
        assert "import oracle" not in src and "from oracle" not in src, f
