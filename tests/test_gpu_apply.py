"""The variational MPO-MPS product (Sect. 2.4.2, matrix-vector product; apply
mode of seemps_sweep) and its two new C-ABI calls vs the oracle:

- seemps_env_update_braket: the environments of <x, W b> element by element
  (left and right, ragged bonds, x and b of different bond dimension);
- seemps_heff_apply_braket: the pair's MPO action between x's and b's bonds;
- the apply sweep: dense states and distances against the oracle's
  apply_mpo (FP64 1e-9), the exact product W b when the bond suffices, and
  the mixed-precision split on large pair matrices (1e-5 of |W b|^2).
"""
import numpy as np
import pytest

import workloads as wl
from oracle import sweep as S

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-11
MIXED_TOL = 2e-4  # bf16x3 products: relative error near 2^-16 per product


@pytest.fixture(scope="module")
def pkg():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_2601_16734_gb300 as pkg
    pkg.build()
    return pkg


@pytest.fixture(scope="module")
def ctx(pkg):
    c = pkg.Context(0, chi_max=160, d=3, D_max=6, krylov_dim=4, chib_max=160)
    yield c
    assert c.device_status() == 0
    c.close()


def dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def relerr(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def close(a, b, tol):
    """Norm-wise and element-wise (largest error over the largest entry) within tol."""
    assert relerr(a, b) < tol, relerr(a, b)
    assert np.abs(a - b).max() <= tol * max(np.abs(b).max(), 1e-300), np.abs(a - b).max() / np.abs(b).max()


ENV_SHAPES = [  # cix, cib, cox, cob, d, Di, Do
    (1, 1, 2, 3, 2, 1, 3), (5, 7, 6, 4, 2, 3, 3), (33, 17, 40, 21, 3, 2, 4), (64, 96, 64, 128, 2, 5, 5),
    (70, 129, 66, 100, 2, 4, 5),
]


@pytest.mark.parametrize("shape", ENV_SHAPES)
@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_env_update_braket(ctx, pkg, shape, prec):
    cix, cib, cox, cob, d, Di, Do = shape
    rng = np.random.default_rng(sum(shape))
    p = pkg.FP64 if prec == "fp64" else pkg.BF16X3
    tol = FP64_TOL if prec == "fp64" else MIXED_TOL
    E = rng.standard_normal((cix, Di, cib))
    W = rng.standard_normal((Di, d, d, Do))
    X = rng.standard_normal((cix, d, cox))
    B = rng.standard_normal((cib, d, cob))
    out = host(ctx.env_update_braket(pkg.LEFT, dev(E), dev(X), dev(B), dev(W), precision=p))
    close(out, S.left_env_mixed(E, X, W, B), tol)
    # right: E (cix, Di, cib) with W (Do, d, d, Di), X (cox, d, cix), B (cob, d, cib)
    Wr = rng.standard_normal((Do, d, d, Di))
    Xr = rng.standard_normal((cox, d, cix))
    Br = rng.standard_normal((cob, d, cib))
    out = host(ctx.env_update_braket(pkg.RIGHT, dev(E), dev(Xr), dev(Br), dev(Wr), precision=p))
    close(out, S.right_env_mixed(E, Xr, Wr, Br), tol)


HEFF_SHAPES = [  # chi_l, chi_r, chib_l, chib_r, d, D_l, D_m, D_r
    (1, 4, 1, 8, 2, 1, 5, 5), (7, 3, 9, 5, 2, 3, 3, 3), (40, 44, 60, 20, 2, 5, 5, 5), (33, 17, 12, 64, 3, 2, 4, 3),
    (96, 128, 128, 96, 2, 5, 4, 5),
]


@pytest.mark.parametrize("shape", HEFF_SHAPES)
@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_heff_apply_braket(ctx, pkg, shape, prec):
    chl, chr_, cbl, cbr, d, Dl, Dm, Dr = shape
    rng = np.random.default_rng(sum(shape) + 1)
    L = rng.standard_normal((chl, Dl, cbl))
    R = rng.standard_normal((chr_, Dr, cbr))
    W1 = rng.standard_normal((Dl, d, d, Dm))
    W2 = rng.standard_normal((Dm, d, d, Dr))
    th = rng.standard_normal((cbl, d, d, cbr))
    p = pkg.FP64 if prec == "fp64" else pkg.BF16X3
    y = host(ctx.heff_apply_braket(dev(L), dev(W1), dev(W2), dev(R), dev(th), precision=p))
    assert y.shape == (chl, d, d, chr_)
    close(y, S.heff_apply(L, W1, W2, R, th), (FP64_TOL if prec == "fp64" else MIXED_TOL))


def _apply(pkg, W, b, x0, chi, n_sweeps, precision):
    chib = max(t.shape[2] for t in b)
    D = max(w.shape[3] for w in W)
    ctx = pkg.Context(0, chi_max=chi, d=b[0].shape[1], D_max=D, krylov_dim=2, chib_max=chib)
    try:
        ch = pkg.Chain(ctx, W, x0, chi, B=b)
        rep = ctx.sweep(ch, mode=pkg.MODE_APPLY, n_sweeps=n_sweeps, precision=precision, chi_max=chi, tol=1e-30)
        x = [host(t) for t in ch.tensors()]
        assert ctx.device_status() == 0
    finally:
        ctx.close()
    return rep, x


def _dense(A):
    return S.mps_to_dense(A).reshape(-1)


def test_apply_fp64_matches_oracle(pkg):
    n, chib, chi = 12, 10, 12
    W = wl.mpo.xxz(n, 0.7)
    b = wl.states.random_mps(n, 2, chib, 71)
    x0 = wl.states.random_mps(n, 2, chi, 72)
    rep, x = _apply(pkg, W, b, x0, chi, 2, pkg.FP64)
    xo, log = S.apply_mpo(W, b, x0, chi, 1e-30, 2)
    ub = S.mpo_to_dense(W) @ _dense(b)
    nu = ub @ ub
    d_gpu, d_or = np.sum((_dense(x) - ub) ** 2), np.sum((_dense(xo) - ub) ** 2)
    assert d_or > 1e-6 * nu
    assert abs(d_gpu - d_or) <= 1e-10 * nu
    assert np.linalg.norm(_dense(x) - _dense(xo)) <= 1e-9 * np.sqrt(nu)
    assert max(a.shape[2] for a in x) <= chi
    assert abs(rep["error_bound"] - log.error) <= 1e-6 * log.error


def test_apply_exact_with_enough_bond(pkg):
    n, chib = 10, 4
    W = wl.mpo.tfim(n, 0.9)
    b = wl.states.random_mps(n, 2, chib, 73)
    x0 = wl.states.random_mps(n, 2, 3, 74)
    _, x = _apply(pkg, W, b, x0, 3 * chib, 2, pkg.FP64)
    ub = S.mpo_to_dense(W) @ _dense(b)
    assert np.linalg.norm(_dense(x) - ub) <= 1e-11 * np.linalg.norm(ub)


def test_apply_mixed_split_large_bond(pkg):
    """b of bond 120 on 14 sites through XXZ (D = 5) compressed to bond 80:
    the pair matrices reach 160 x 160, so the mixed split runs the FP32 QR +
    block Jacobi path; distances agree with the oracle to 1e-5 of |W b|^2."""
    n, chib, chi = 14, 120, 80
    W = wl.mpo.xxz(n, 1.0)
    b = wl.states.random_mps(n, 2, chib, 75)
    b = [t / np.sqrt(t.shape[0] * t.shape[1]) for t in b]
    x0 = wl.states.random_mps(n, 2, chi, 76)
    _, x = _apply(pkg, W, b, x0, chi, 2, pkg.BF16X3)
    _, x64 = _apply(pkg, W, b, x0, chi, 2, pkg.FP64)
    xo, _ = S.apply_mpo(W, b, x0, chi, 1e-30, 2)
    C = S.mpo_mps_product(W, b)
    nu = S.overlap(C, C)
    d_or = S.distance2(xo, C)
    assert d_or > 1e-6 * nu
    assert abs(S.distance2(x64, C) - d_or) <= 1e-10 * nu
    assert abs(S.distance2(x, C) - d_or) <= 1e-5 * nu
    assert S.distance2(x, xo) <= 1e-5 * nu


def test_apply_rejects_chain_without_b(pkg):
    from paper_2601_16734_gb300 import abi
    ctx = pkg.Context(0, chi_max=4, d=2, D_max=3, krylov_dim=2)
    try:
        ch = pkg.Chain(ctx, wl.mpo.tfim(4, 1.0), wl.states.random_mps(4, 2, 4, 1), 4)
        with pytest.raises(abi.SeempsError) as e:
            ctx.sweep(ch, mode=pkg.MODE_APPLY, chi_max=4)
        assert e.value.status == 1
        assert ctx.device_status() == 0
    finally:
        ctx.close()
