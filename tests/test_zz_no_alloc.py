"""The allocation-free effective-operator apply (seemps_heff_apply_noalloc).

Some callers cannot allocate device memory (their memory belongs to an
allocator that will not hand them a buffer, or they must not allocate at
all), so they cannot provide the workspace the other entry points need.
This test calls the allocation-free entry point through the C ABI twice in a
row and checks each result against the workspace-based seemps_heff_apply
(FP64) at the FP64 tolerance of the parity tests; it also checks that sizes
beyond the static scratch are refused before anything runs.  It lives in a
file pytest collects last and depends on no state left by other tests.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-11


def _inputs(rng, chl, chr_, d, Dl, Dm, Dr):
    return (rng.standard_normal((chl, Dl, chl)), rng.standard_normal((Dl, d, d, Dm)),
            rng.standard_normal((Dm, d, d, Dr)), rng.standard_normal((chr_, Dr, chr_)),
            rng.standard_normal((chl, d, d, chr_)))


def test_noalloc_matches_workspace_apply_twice():
    import torch
    import paper_2601_16734_gb300 as pkg
    from paper_2601_16734_gb300 import abi

    assert torch.cuda.is_available()
    pkg.build()
    lib = abi.load()
    ctx = pkg.Context(0, chi_max=128, d=2, D_max=5)
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    err = ctypes.create_string_buffer(512)
    rng = np.random.default_rng(2024)
    for shape in ((37, 61, 2, 5, 5, 5), (96, 96, 2, 3, 5, 1)):
        L, W1, W2, R, th = (dev(x) for x in _inputs(rng, *shape))
        ref = ctx.heff_apply(L, W1, W2, R, th, precision=pkg.FP64)
        dims = abi.PairDims(*shape[:2], shape[2], *shape[3:])
        for call in range(2):  # two calls in a row share the static scratch
            y = torch.full_like(th, float("nan"))
            st = lib.seemps_heff_apply_noalloc(ctypes.byref(dims), L.data_ptr(), W1.data_ptr(),
                                               W2.data_ptr(), R.data_ptr(), th.data_ptr(),
                                               y.data_ptr(), stream, err, len(err))
            assert st == 0, err.value.decode()
            torch.cuda.synchronize()
            rel = (torch.linalg.vector_norm(y - ref) / torch.linalg.vector_norm(ref)).item()
            assert rel < FP64_TOL, (shape, call, rel)
    # one shape against the CPU oracle's index sum as well (independent of the
    # workspace path's plan and kernels)
    from oracle import sweep as S
    Ln, W1n, W2n, Rn, thn = _inputs(np.random.default_rng(7), 29, 33, 2, 5, 5, 5)
    dims = abi.PairDims(29, 33, 2, 5, 5, 5)
    L, W1, W2, R, th = (dev(x) for x in (Ln, W1n, W2n, Rn, thn))  # kept alive across the call
    y = torch.full_like(th, float("nan"))
    st = lib.seemps_heff_apply_noalloc(ctypes.byref(dims), L.data_ptr(), W1.data_ptr(), W2.data_ptr(),
                                       R.data_ptr(), th.data_ptr(), y.data_ptr(), stream, err, len(err))
    assert st == 0, err.value.decode()
    torch.cuda.synchronize()
    ref = S.heff_apply(Ln, W1n, W2n, Rn, thn)
    assert np.linalg.norm(y.cpu().numpy() - ref) < FP64_TOL * np.linalg.norm(ref)
    assert ctx.device_status() == 0
    ctx.close()


def test_noalloc_rejects_oversize():
    import torch
    from paper_2601_16734_gb300 import abi

    lib = abi.load()
    dims = abi.PairDims(1024, 1024, 2, 5, 5, 5)  # intermediates ~335 MB > 32 MiB
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    y = torch.zeros(8, dtype=torch.float64, device="cuda")
    err = ctypes.create_string_buffer(512)
    st = lib.seemps_heff_apply_noalloc(ctypes.byref(dims), x.data_ptr(), x.data_ptr(), x.data_ptr(),
                                       x.data_ptr(), x.data_ptr(), y.data_ptr(), None, err, len(err))
    assert st == 3  # SEEMPS_ERR_WORKSPACE
    assert b"maximum" in err.value
    # sizes whose byte counts would wrap a 64-bit integer are refused too
    dims = abi.PairDims(1 << 30, 1 << 30, 2, 1, 1, 1)
    st = lib.seemps_heff_apply_noalloc(ctypes.byref(dims), x.data_ptr(), x.data_ptr(), x.data_ptr(),
                                       x.data_ptr(), x.data_ptr(), y.data_ptr(), None, err, len(err))
    assert st == 1  # SEEMPS_ERR_INVALID: dimension out of range
