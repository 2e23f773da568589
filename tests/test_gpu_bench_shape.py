"""Parity at the benchmark's shape: the bulk pair of an XXZ chain at chi = 1024
(Delta = 1, D = 5, d = 2, Lanczos dimension 20), the launch configuration
that bench.py times, GPU (through the C ABI) against the CPU oracle on
identical inputs.

The environments are the oracle's own contraction of the XXZ MPO with seeded
random isometries (QR of Gaussian matrices on the CPU): a 22-site chain whose
middle bonds reach 1024, so that L_10 and R_12 are genuine chi = 1024
quadratic-form environments and H_n is symmetric.  Every comparison is
element-wise (largest error over the largest entry) as well as norm-wise.
At this shape the first GEMM of H_n (M = chi D = 5120, N = d^2 chi = 4096)
runs on 128 x 256 tensor-core tiles; a ragged directed shape below selects
the same tiles with partial tiles on every edge.
"""
import numpy as np
import pytest

import workloads as wl
from oracle import sweep as S

pytestmark = pytest.mark.gpu

N_SITES, PAIR, CHI = 22, 10, 1024
FP64_TOL = 1e-11
MIXED_TOL = 1e-4  # bf16x3: ~2^-16 per product, FP32 accumulation
ENV_MIXED_TOL = 1e-5  # six products from three bf16 planes, four accumulators per output


def bond(k):
    return min(2 ** k, 2 ** (N_SITES - k), CHI)


@pytest.fixture(scope="module")
def pkg():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_2601_16734_gb300 as pkg
    pkg.build()
    return pkg


@pytest.fixture(scope="module")
def ctx(pkg):
    c = pkg.Context(0, chi_max=CHI, d=2, D_max=5, krylov_dim=20)
    yield c
    assert c.device_status() == 0
    c.close()


@pytest.fixture(scope="module")
def pair():
    """CPU-built inputs of the pair (PAIR, PAIR + 1) and the oracle's results."""
    rng = np.random.default_rng(2024)
    W = wl.mpo.xxz(N_SITES, 1.0)
    L = np.ones((1, 1, 1))
    for k in range(PAIR):
        chl, chr_ = bond(k), bond(k + 1)
        Q = np.linalg.qr(rng.standard_normal((chl * 2, chr_)))[0]
        L = S.left_env(L, Q.reshape(chl, 2, chr_), W[k])
    R = np.ones((1, 1, 1))
    for k in range(N_SITES - 1, PAIR + 1, -1):
        chl, chr_ = bond(k), bond(k + 1)
        Q = np.linalg.qr(rng.standard_normal((2 * chr_, chl)))[0]
        R = S.right_env(R, Q.T.reshape(chl, 2, chr_), W[k])
    assert L.shape == (CHI, 5, CHI) and R.shape == (CHI, 5, CHI)
    theta = rng.standard_normal((CHI, 2, 2, CHI))
    theta /= np.linalg.norm(theta)
    W1, W2 = W[PAIR], W[PAIR + 1]
    mv = lambda v: S.heff_apply(L, W1, W2, R, v)  # noqa: E731
    y = mv(theta)
    E, theta_star, m = S.lanczos_lowest(mv, theta, 20)
    # a left isometry for the environment update across site PAIR
    A = np.linalg.qr(rng.standard_normal((CHI * 2, CHI)))[0].reshape(CHI, 2, CHI)
    return dict(W1=W1, W2=W2, L=L, R=R, theta=theta, y=y, E=E, theta_star=theta_star, m=m, A=A,
                L_next=S.left_env(L, A, W1))


def dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def check(a, b, tol, what):
    nerr = np.linalg.norm(a - b) / np.linalg.norm(b)
    eerr = np.abs(a - b).max() / np.abs(b).max()
    print(f"{what}: norm-wise {nerr:.2e}, element-wise {eerr:.2e} (bound {tol:.0e})")
    assert nerr <= tol and eerr <= tol


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_heff_apply_chi1024(ctx, pkg, pair, prec):
    p, tol = (pkg.FP64, FP64_TOL) if prec == "fp64" else (pkg.BF16X3, MIXED_TOL)
    y = ctx.heff_apply(dev(pair["L"]), dev(pair["W1"]), dev(pair["W2"]), dev(pair["R"]), dev(pair["theta"]),
                       precision=p)
    check(host(y), pair["y"], tol, f"H_n theta at chi=1024 ({prec})")


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_env_update_chi1024(ctx, pkg, pair, prec):
    # the mixed environment update forms six bf16 products (three planes, ~2^-24 each); at
    # K = 1024 and 2048 the tensor cores' FP32 accumulation sets the error: one accumulator
    # per output gave 1.9e-5 here (against 2.4e-7 for an IEEE-rounded emulation), the four
    # interleaved accumulators of the six-product GEMM 4.8e-6
    p, tol = (pkg.FP64, FP64_TOL) if prec == "fp64" else (pkg.BF16X3, ENV_MIXED_TOL)
    out = ctx.env_update(pkg.LEFT, dev(pair["L"]), dev(pair["A"]), dev(pair["W1"]), precision=p)
    check(host(out), pair["L_next"], tol, f"L_11 at chi=1024 ({prec})")


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_lanczos_energy_chi1024(ctx, pkg, pair, prec):
    """Same start vector, Krylov dimension 20: the lowest Ritz value.  FP64
    to 1e-10 relative; bf16x3 (operator error ~2^-16 per product) to 1e-4 of
    the spectral scale, as in the smaller mixed Lanczos parity test."""
    p = pkg.FP64 if prec == "fp64" else pkg.BF16X3
    t = dev(pair["theta"])
    e, m = ctx.local_eig(dev(pair["L"]), dev(pair["W1"]), dev(pair["W2"]), dev(pair["R"]), t, krylov_dim=20,
                         precision=p)
    E = pair["E"]
    print(f"Lanczos at chi=1024 ({prec}): {e!r} vs oracle {E!r}, rel {abs(e - E) / abs(E):.2e}")
    assert m == pair["m"]
    assert abs(e - E) <= (1e-10 if prec == "fp64" else 1e-4) * abs(E)
    if prec == "fp64":
        assert abs(abs(float(np.sum(host(t) * pair["theta_star"]))) - 1.0) <= 1e-8


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_split_singular_values_chi1024(ctx, pkg, pair, prec):
    """The split of the Lanczos vector as a 2048 x 2048 matrix: singular values
    against LAPACK.  Both are backward stable, so they agree to a few n eps s_0
    (n = 2048: n eps = 4.5e-13); the FP64 Jacobi is held to 1e-12 s_0, the
    mixed split (FP32 rotations) to 1e-4 s_0."""
    p = pkg.FP64 if prec == "fp64" else pkg.BF16X3
    M = pair["theta_star"].reshape(CHI * 2, 2 * CHI)
    res = ctx.svd_truncate(dev(M), CHI, 1e-12, absorb=pkg.ABSORB_RIGHT, normalize=True, precision=p)
    s_ref = np.linalg.svd(M, compute_uv=False)
    err = np.abs(host(res.S) - s_ref).max() / s_ref[0]
    print(f"split at chi=1024 ({prec}): max |s - s_LAPACK| = {err:.2e} s_0, rank {res.rank}")
    assert err <= (1e-12 if prec == "fp64" else 1e-4)
    assert res.rank == S.truncation_rank(host(res.S), CHI, 1e-12)


def _sym_env(rng, chi, D):
    L = rng.standard_normal((chi, D, chi))
    return 0.5 * (L + L.transpose(2, 1, 0))


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_heff_apply_ragged_wide_tiles(ctx, pkg, prec):
    """chi_l = 700, chi_r = 650: the first GEMM (M = 3500, N = 2600) has 308
    tiles of 128 x 256, above the 1.5 waves that select them, and every edge
    (M, N and K = 700) ends in a partial tile."""
    rng = np.random.default_rng(700)
    W = wl.mpo.xxz(4, 1.0)
    L, R = _sym_env(rng, 700, 5), _sym_env(rng, 650, 5)
    th = rng.standard_normal((700, 2, 2, 650))
    p, tol = (pkg.FP64, FP64_TOL) if prec == "fp64" else (pkg.BF16X3, MIXED_TOL)
    y = host(ctx.heff_apply(dev(L), dev(W[1]), dev(W[2]), dev(R), dev(th), precision=p))
    check(y, S.heff_apply(L, W[1], W[2], R, th), tol, f"H_n theta at 700 x 650 ({prec})")


@pytest.mark.parametrize("shape", [(1024, 1024, 5, 5), (700, 650, 5, 5), (333, 257, 3, 5), (64, 96, 5, 3)])
def test_fused_mixing_is_bit_identical(ctx, pkg, shape):
    """The MPO mixing done in the first GEMM's epilogue (tiles of whole D_l
    row groups, theta's columns reordered to (c, s)) against the separate
    mixing kernel: the same FP32 products and sums in the same order, so the
    outputs agree bit for bit; both against the oracle at the bf16x3 bound."""
    cl, cr, Dl, Dr = shape
    rng = np.random.default_rng(cl + cr)
    W = wl.mpo.xxz(4, 1.0)
    W1 = W[1][:Dl] if Dl < 5 else W[1]
    W2 = W[2][:, :, :, :Dr] if Dr < 5 else W[2]
    L, R = _sym_env(rng, cl, W1.shape[0]), _sym_env(rng, cr, W2.shape[3])
    th = rng.standard_normal((cl, 2, 2, cr))
    args = (dev(L), dev(W1), dev(W2), dev(R), dev(th))
    ctx.set_fused_mixing(False)
    y_sep = host(ctx.heff_apply(*args, precision=pkg.BF16X3))
    ctx.set_fused_mixing(True)
    y_fused = host(ctx.heff_apply(*args, precision=pkg.BF16X3))
    assert np.array_equal(y_sep, y_fused)
    check(y_fused, S.heff_apply(L, W1, W2, R, th), MIXED_TOL, f"fused H_n theta at {cl} x {cr}, D {Dl}/{Dr}")
