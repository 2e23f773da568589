"""Variational compression (simplify mode of seemps_sweep) vs the oracle's
simplify: the same target b, the same initial guess, the same strategy.

The compressed state is unique up to gauge, so dense vectors (small N) and
distances |x - b|^2 (from overlaps) are compared: FP64 to 1e-10 relative,
the mixed-precision split (FP32 QR + Jacobi) to 1e-5 of |b|^2.
"""
import numpy as np
import pytest

import workloads as wl
from oracle import sweep as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_2601_16734_gb300 as pkg
    pkg.build()
    return pkg


def _run(pkg, b, x0, chi, n_sweeps, precision, chib):
    ctx = pkg.Context(0, chi_max=chi, d=b[0].shape[1], D_max=1, krylov_dim=2, chib_max=chib)
    try:
        ch = pkg.Chain(ctx, None, x0, chi, B=b)
        rep = ctx.sweep(ch, mode=pkg.MODE_SIMPLIFY, n_sweeps=n_sweeps, precision=precision, chi_max=chi,
                        tol=1e-30)
        x = [t.detach().cpu().numpy() for t in ch.tensors()]
        assert ctx.device_status() == 0
    finally:
        ctx.close()
    return rep, x


def test_simplify_fp64_matches_oracle(pkg):
    n, chib, chi = 12, 24, 10
    b = wl.states.random_mps(n, 2, chib, 31)
    x0 = wl.states.random_mps(n, 2, chi, 32)
    rep, x = _run(pkg, b, x0, chi, 2, pkg.FP64, chib)
    xo, _ = S.simplify(b, x0, chi, 1e-30, 2)
    nb = S.overlap(b, b)
    d_gpu, d_or = S.distance2(x, b), S.distance2(xo, b)
    assert d_or > 1e-6 * nb
    assert abs(d_gpu - d_or) <= 1e-10 * nb
    v, vo = S.mps_to_dense(x).reshape(-1), S.mps_to_dense(xo).reshape(-1)
    assert np.linalg.norm(v - vo) <= 1e-9 * np.sqrt(nb)
    assert max(a.shape[2] for a in x) <= chi
    assert rep["error_bound"] > 0.0


def test_simplify_exact_with_enough_bond(pkg):
    n, chib = 12, 24
    b = wl.states.random_mps(n, 2, chib, 41)
    x0 = wl.states.random_mps(n, 2, 4, 42)
    _, x = _run(pkg, b, x0, chib, 2, pkg.FP64, chib)
    v, vb = S.mps_to_dense(x).reshape(-1), S.mps_to_dense(b).reshape(-1)
    assert np.linalg.norm(v - vb) <= 1e-11 * np.linalg.norm(vb)


def test_simplify_mixed_split_large_bond(pkg):
    """Bond 160 -> 70 on 16 sites (relative residual ~4e-4): the pair
    matrices reach 140 x 140, so the mixed split runs the FP32 QR + block
    Jacobi path; its result agrees with the FP64 optimum to 1e-5 of |b|^2."""
    n, chib, chi = 16, 160, 70
    b = wl.states.random_mps(n, 2, chib, 51)
    x0 = wl.states.random_mps(n, 2, chi, 52)
    _, x = _run(pkg, b, x0, chi, 2, pkg.BF16X3, chib)
    _, x64 = _run(pkg, b, x0, chi, 2, pkg.FP64, chib)
    xo, _ = S.simplify(b, x0, chi, 1e-30, 2)
    nb = S.overlap(b, b)
    d_or = S.distance2(xo, b)
    assert d_or > 1e-4 * nb
    assert abs(S.distance2(x64, b) - d_or) <= 1e-10 * nb
    assert abs(S.distance2(x, b) - d_or) <= 1e-5 * nb
    assert S.distance2(x, xo) <= 1e-5 * nb
