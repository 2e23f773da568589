"""Edge cases of the C ABI on the GPU: refused arguments come back as status
codes (never a fault), degenerate splits stay finite, the Lanczos handles a
Krylov dimension above the local dimension, and the mixed split's largest
shapes (isometric side up to 4096 rows, QR input up to 4096 rows) agree
with LAPACK."""
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


@pytest.fixture(scope="module")
def ctx(pkg):
    c = pkg.Context(0, chi_max=64, d=2, D_max=5, krylov_dim=24, chib_max=16)
    yield c
    assert c.device_status() == 0
    c.close()


def dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def test_refused_arguments_are_status_codes(ctx, pkg):
    from paper_2601_16734_gb300 import abi
    with pytest.raises(abi.SeempsError) as e:
        ctx.svd_truncate(dev(np.zeros((0, 4))), 4, 1e-12)
    assert e.value.status == 1
    with pytest.raises(abi.SeempsError) as e:
        ctx.svd_truncate(dev(np.ones((4, 4))), 0, 1e-12)  # chi_max < 1
    assert e.value.status == 1
    L, R = dev(np.ones((4, 1, 4))), dev(np.ones((4, 1, 4)))
    W = dev(np.ones((1, 2, 2, 1)))
    th = dev(np.ones((4, 2, 2, 4)))
    with pytest.raises(abi.SeempsError) as e:
        ctx.local_eig(L, W, W, R, th, krylov_dim=1000)  # above the largest Krylov dimension
    assert e.value.status == 1
    with pytest.raises(abi.SeempsError) as e:
        ctx.env_update(7, L, dev(np.ones((4, 2, 4))), W)  # no such side
    assert e.value.status == 1
    # an MPS without b in solve mode, an unknown mode
    n = 4
    ch = pkg.Chain(ctx, wl.mpo.tfim(n, 1.0), wl.states.random_mps(n, 2, 4, 1), 4)
    with pytest.raises(abi.SeempsError) as e:
        ctx.sweep(ch, mode=pkg.MODE_SOLVE, chi_max=4)
    assert e.value.status == 1
    with pytest.raises(abi.SeempsError) as e:
        ctx.sweep(ch, mode=9, chi_max=4)
    assert e.value.status == 1
    assert ctx.device_status() == 0


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
@pytest.mark.parametrize("shape", [(1, 1), (1, 7), (7, 1), (300, 300)])
def test_zero_matrix_split(ctx, pkg, prec, shape):
    """theta = 0: rank 1, zero factors, no NaN, zero discarded weight."""
    p = pkg.FP64 if prec == "fp64" else pkg.BF16X3
    m, n = shape
    res = ctx.svd_truncate(dev(np.zeros((m, n))), 8, 1e-12, precision=p)
    assert res.rank == 1
    for t in (res.A_left, res.A_right, res.S):
        v = host(t)
        assert np.isfinite(v).all()
    assert np.abs(host(res.A_left) @ host(res.A_right)).max() == 0.0
    assert res.discarded == 0.0


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_vector_shaped_splits(ctx, pkg, prec):
    """1 x n and m x 1 two-site matrices: one singular value, |M|."""
    p = pkg.FP64 if prec == "fp64" else pkg.BF16X3
    tol = 1e-12 if prec == "fp64" else 1e-6  # the mixed split's column norms come from FP32 data
    rng = np.random.default_rng(4)
    for shape in ((1, 9), (9, 1)):
        M = rng.standard_normal(shape)
        res = ctx.svd_truncate(dev(M), 4, 1e-12, precision=p)
        assert res.rank == 1
        assert abs(host(res.S)[0] - np.linalg.norm(M)) <= tol * np.linalg.norm(M)
        assert np.abs(host(res.A_left) @ host(res.A_right) - M).max() <= tol * np.abs(M).max()


def test_lanczos_krylov_above_local_dimension(ctx, pkg):
    """n_loc = 16 < krylov_dim = 20: the exact lowest eigenvalue of H_n."""
    W = wl.mpo.xxz(4, 1.0)
    A = wl.states.random_mps(4, 2, 2, 3)
    Lenv = S.left_env(np.ones((1, 1, 1)), A[0], W[0])
    Renv = S.right_env(np.ones((1, 1, 1)), A[3], W[3])
    th = S.two_site(A[1], A[2])
    Hd = S.heff_dense(Lenv, W[1], W[2], Renv)
    e_exact = np.linalg.eigvalsh(0.5 * (Hd + Hd.T))[0]
    e, it = ctx.local_eig(dev(Lenv), dev(W[1]), dev(W[2]), dev(Renv), dev(th), krylov_dim=20)
    assert it <= th.size
    assert abs(e - e_exact) <= 1e-11 * max(1.0, abs(e_exact))


@pytest.mark.parametrize("m,n,absorb", [(3000, 2000, "right"), (2000, 3000, "right"), (2000, 3000, "left")])
def test_mixed_split_largest_shapes(pkg, m, n, absorb):
    """Isometric side 3000 long (the 4-column-block Jacobi kernel) or a QR
    input of 3000 rows (the 8-column panel kernel)."""
    ctx = pkg.Context(0, chi_max=1500, d=2, D_max=1, krylov_dim=2)
    try:
        rng = np.random.default_rng(m + 3 * n)
        p = min(m, n)
        M = rng.standard_normal((m, p)) @ np.diag(np.exp(-np.arange(p) / 200.0)) @ \
            np.linalg.qr(rng.standard_normal((n, p)))[0].T
        ab = pkg.ABSORB_RIGHT if absorb == "right" else pkg.ABSORB_LEFT
        res = ctx.svd_truncate(dev(M), p // 2, 1e-12, absorb=ab, precision=pkg.BF16X3)
        s_ref = np.linalg.svd(M, compute_uv=False)
        assert np.abs(host(res.S)[:p] - s_ref).max() <= 1e-4 * s_ref[0]
        iso = host(res.A_left) if ab == pkg.ABSORB_RIGHT else host(res.A_right).T
        assert np.abs(iso.T @ iso - np.eye(res.rank)).max() < 1e-4
        assert ctx.device_status() == 0
    finally:
        ctx.close()
