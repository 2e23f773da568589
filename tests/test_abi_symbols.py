"""The C-ABI library builds for sm_103a and exports every declared entry point
(runs on the CPU: no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            text = open(os.path.join(inc, f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(seemps_[a-z_0-9]+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_2601_16734_gb300 import _build
    return ctypes.CDLL(_build.lib_path())


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("seemps_env_update", "seemps_heff_apply", "seemps_local_eig",
                     "seemps_local_pcg", "seemps_svd_truncate", "seemps_sweep"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_the_header():
    from paper_2601_16734_gb300 import abi
    covered = set(abi._SIGS) | {"seemps_last_error"}
    assert set(_declared()) <= covered


def test_create_rejects_bad_workspace_without_gpu(lib):
    # argument checks run before any CUDA call
    h = ctypes.c_void_p()
    lib.seemps_create.restype = ctypes.c_int
    assert lib.seemps_create(ctypes.byref(h), 0, None, None, ctypes.c_size_t(0)) == 1
