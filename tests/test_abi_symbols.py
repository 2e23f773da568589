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


def test_host_size_queries_without_gpu(lib):
    """The host-only size queries: positive, growing with the bond limit, and
    refusing bad arguments with SEEMPS_ERR_INVALID."""
    ws = ctypes.c_size_t(0)
    lib.seemps_workspace_bytes.restype = ctypes.c_int
    lib.seemps_cgs_work_bytes.restype = ctypes.c_int
    sizes = []
    for chi in (16, 64, 256):
        assert lib.seemps_workspace_bytes(chi, 2, 5, 20, 2 * chi, ctypes.byref(ws)) == 0
        sizes.append(ws.value)
    assert 0 < sizes[0] < sizes[1] < sizes[2]
    cg = []
    for chi in (8, 32, 128):
        assert lib.seemps_cgs_work_bytes(24, 2, 3, chi, 16, ctypes.byref(ws)) == 0
        cg.append(ws.value)
    assert 0 < cg[0] < cg[1] < cg[2]
    # at bond 64 on 24 sites: three work MPS, one joined MPS of bond 128, 50 environments
    assert lib.seemps_cgs_work_bytes(24, 2, 3, 64, 16, ctypes.byref(ws)) == 0
    need = 24 * (3 * 64 * 2 * 64 + 128 * 2 * 128) * 8 + 50 * max(64 * 128, 64 * 3 * 64) * 8
    assert need <= ws.value <= need + 200 * 256 + 256
    assert lib.seemps_cgs_work_bytes(1, 2, 3, 64, 16, ctypes.byref(ws)) == 1  # one site
    assert lib.seemps_cgs_work_bytes(24, 2, 3, 0, 16, ctypes.byref(ws)) == 1  # chi_max 0
    assert lib.seemps_cgs_work_bytes(24, 2, 3, 64, 16, None) == 1
