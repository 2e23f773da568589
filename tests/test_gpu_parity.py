"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerances: FP64 kernels agree with the FP64 oracle to rounding (1e-11
relative, a few hundred ulps of accumulated reordering); bf16x3 products
carry a relative error near 2^-16 per product, so norm-wise 2e-4 bounds them
with margin.  Truncation ranks are compared exactly.
"""
import numpy as np
import pytest

import workloads as wl
from oracle import exact as X
from oracle import sweep as S

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-11
MIXED_TOL = 2e-4
ENV_MIXED_TOL = 5e-6


@pytest.fixture(scope="module")
def pkg():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_2601_16734_gb300 as pkg
    pkg.build()
    return pkg


@pytest.fixture(scope="module")
def ctx(pkg):
    c = pkg.Context(0, chi_max=160, d=3, D_max=6, krylov_dim=24, chib_max=16)
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
    """Norm-wise relative error and the largest element-wise error over the
    largest entry both within tol (a wrong tail tile or a few bad elements
    cannot hide under the norm)."""
    assert relerr(a, b) < tol, relerr(a, b)
    assert np.abs(a - b).max() <= tol * max(np.abs(b).max(), 1e-300), np.abs(a - b).max() / np.abs(b).max()


SHAPES = [  # chi_l, chi_r, d, D_l, D_m, D_r
    (1, 1, 2, 1, 3, 1), (1, 4, 2, 1, 5, 5), (3, 7, 2, 3, 3, 3), (16, 16, 2, 5, 5, 5),
    (33, 17, 3, 2, 4, 3), (64, 64, 2, 5, 5, 5), (130, 66, 2, 3, 5, 1), (97, 129, 2, 5, 3, 5),
    (40, 44, 2, 6, 4, 6), (48, 20, 3, 3, 3, 2),  # mixing blocks of 24 and 27 inputs
    (64, 48, 2, 20, 23, 26), (40, 40, 2, 12, 10, 14),  # wide blocks: 80 -> 104 and 48 -> 56 (J1-J2 bonds)
]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_heff_apply(ctx, pkg, shape, prec):
    chl, chr_, d, Dl, Dm, Dr = shape
    rng = np.random.default_rng(sum(shape))
    L = rng.standard_normal((chl, Dl, chl))
    W1 = rng.standard_normal((Dl, d, d, Dm))
    W2 = rng.standard_normal((Dm, d, d, Dr))
    R = rng.standard_normal((chr_, Dr, chr_))
    th = rng.standard_normal((chl, d, d, chr_))
    p = pkg.FP64 if prec == "fp64" else pkg.BF16X3
    y = host(ctx.heff_apply(dev(L), dev(W1), dev(W2), dev(R), dev(th), precision=p))
    ref = S.heff_apply(L, W1, W2, R, th)
    close(y, ref, (FP64_TOL if prec == "fp64" else MIXED_TOL))


ENV_SHAPES = [(1, 2, 2, 1, 3), (4, 8, 2, 3, 3), (7, 5, 3, 2, 4), (33, 64, 2, 5, 5), (129, 70, 2, 5, 3),
              (64, 48, 2, 6, 5), (36, 44, 3, 3, 4), (40, 48, 2, 26, 23),
              (1100, 64, 2, 5, 5)]  # long K over few output tiles: the split-K path


@pytest.mark.parametrize("shape", ENV_SHAPES)
@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_env_update(ctx, pkg, shape, prec):
    ci, co, d, Di, Do = shape
    rng = np.random.default_rng(7 * ci + co)
    p = pkg.FP64 if prec == "fp64" else pkg.BF16X3
    # bf16x3 environment updates split into three planes (six products, ~2^-24 each)
    tol = FP64_TOL if prec == "fp64" else ENV_MIXED_TOL
    E = rng.standard_normal((ci, Di, ci))
    # left: A (ci, d, co), W (Di, d, d, Do)
    A = rng.standard_normal((ci, d, co))
    W = rng.standard_normal((Di, d, d, Do))
    out = host(ctx.env_update(pkg.LEFT, dev(E), dev(A), dev(W), precision=p))
    close(out, S.left_env(E, A, W), tol)
    # right: A (co, d, ci), W (Do, d, d, Di)
    A = rng.standard_normal((co, d, ci))
    W = rng.standard_normal((Do, d, d, Di))
    out = host(ctx.env_update(pkg.RIGHT, dev(E), dev(A), dev(W), precision=p))
    close(out, S.right_env(E, A, W), tol)


@pytest.mark.parametrize("shape", [(1, 3, 1, 2, 2), (9, 5, 4, 3, 2), (64, 32, 12, 20, 2)])
def test_linear_env_and_b_effective(ctx, pkg, shape):
    ci, co, bi, bo, d = shape
    rng = np.random.default_rng(ci + bo)
    F = rng.standard_normal((ci, bi))
    A = rng.standard_normal((ci, d, co))
    B = rng.standard_normal((bi, d, bo))
    out = host(ctx.env_update_linear(pkg.LEFT, dev(F), dev(A), dev(B)))
    close(out, S.left_env_linear(F, A, B), FP64_TOL)
    A2 = rng.standard_normal((co, d, ci))
    B2 = rng.standard_normal((bo, d, bi))
    out = host(ctx.env_update_linear(pkg.RIGHT, dev(F), dev(A2), dev(B2)))
    close(out, S.right_env_linear(F, A2, B2), FP64_TOL)
    G = rng.standard_normal((co, bo))
    B1 = rng.standard_normal((bi, d, 5))
    B2 = rng.standard_normal((5, d, bo))
    out = host(ctx.b_effective(dev(F), dev(B1), dev(B2), dev(G)))
    close(out, S.b_effective(F, B1, B2, G), FP64_TOL)


def test_two_site_and_diagonal(ctx, pkg):
    rng = np.random.default_rng(3)
    A1, A2 = rng.standard_normal((5, 2, 7)), rng.standard_normal((7, 2, 9))
    close(host(ctx.two_site(dev(A1), dev(A2))), S.two_site(A1, A2), FP64_TOL)
    L, W1 = rng.standard_normal((6, 3, 6)), rng.standard_normal((3, 2, 2, 4))
    W2, R = rng.standard_normal((4, 2, 2, 5)), rng.standard_normal((9, 5, 9))
    out = host(ctx.heff_diagonal(dev(L), dev(W1), dev(W2), dev(R)))
    close(out, S.heff_diagonal(L, W1, W2, R), FP64_TOL)


def _sym_env(rng, chi, D):
    """Environment whose H_n is symmetric: L[:, b, :] symmetric for every b."""
    L = rng.standard_normal((chi, D, chi))
    return 0.5 * (L + L.transpose(2, 1, 0))


def _sym_mpo(rng, Dl, d, Dr):
    W = rng.standard_normal((Dl, d, d, Dr))
    return 0.5 * (W + W.transpose(0, 2, 1, 3))


@pytest.mark.parametrize("chi,k", [(2, 16), (6, 20), (24, 20), (60, 12)])
def test_local_eig_matches_oracle(ctx, pkg, chi, k):
    rng = np.random.default_rng(chi)
    d, D = 2, 3
    L, R = _sym_env(rng, chi, D), _sym_env(rng, chi + 1, D)
    W1, W2 = _sym_mpo(rng, D, d, D), _sym_mpo(rng, D, d, D)
    th = rng.standard_normal((chi, d, d, chi + 1))
    mv = lambda v: S.heff_apply(L, W1, W2, R, v)
    e_ref, x_ref, m_ref = S.lanczos_lowest(mv, th, k)
    t = dev(th)
    e, m = ctx.local_eig(dev(L), dev(W1), dev(W2), dev(R), t, krylov_dim=k)
    assert m == m_ref
    assert abs(e - e_ref) <= 1e-10 * max(1.0, abs(e_ref))
    x = host(t)
    assert abs(np.linalg.norm(x) - 1.0) < 1e-12
    assert abs(abs(np.sum(x * x_ref)) - 1.0) < 1e-8
    # Ritz residual equals the oracle's
    r_gpu = np.linalg.norm(mv(x) - e * x)
    r_ref = np.linalg.norm(mv(x_ref) - e_ref * x_ref)
    assert abs(r_gpu - r_ref) <= 1e-8 * max(1.0, abs(e_ref))


@pytest.mark.parametrize("chi", [40, 97])
def test_local_eig_mixed_matches_oracle(ctx, pkg, chi):
    """The bf16x3 sweep's Lanczos (bf16x3 products, FP32 Krylov basis, FP64
    tridiagonal): the operator carries a relative error near 2^-16 per
    product, so the Ritz value agrees with the FP64 oracle to 1e-4 of the
    spectral scale and the Ritz vector's residual under the exact operator
    stays within 1e-3 of that scale of the oracle's."""
    rng = np.random.default_rng(chi + 5)
    d, D = 2, 3
    L, R = _sym_env(rng, chi, D), _sym_env(rng, chi + 3, D)
    W1, W2 = _sym_mpo(rng, D, d, D), _sym_mpo(rng, D, d, D)
    th = rng.standard_normal((chi, d, d, chi + 3))
    mv = lambda v: S.heff_apply(L, W1, W2, R, v)  # noqa: E731
    e_ref, x_ref, m_ref = S.lanczos_lowest(mv, th, 20)
    t = dev(th)
    e, m = ctx.local_eig(dev(L), dev(W1), dev(W2), dev(R), t, krylov_dim=20, precision=pkg.BF16X3)
    assert m == m_ref == 20
    scale = max(1.0, abs(e_ref))
    assert abs(e - e_ref) <= 1e-4 * scale
    x = host(t)
    assert abs(np.linalg.norm(x) - 1.0) < 1e-12  # normalised in FP64
    r_gpu = np.linalg.norm(mv(x) - e_ref * x)
    r_ref = np.linalg.norm(mv(x_ref) - e_ref * x_ref)
    assert r_gpu <= r_ref + 1e-3 * scale


def test_local_eig_full_space_exact(ctx, pkg):
    rng = np.random.default_rng(11)
    L, R = _sym_env(rng, 2, 2), _sym_env(rng, 3, 2)
    W1, W2 = _sym_mpo(rng, 2, 2, 2), _sym_mpo(rng, 2, 2, 2)
    H = S.heff_dense(L, W1, W2, R)
    n = H.shape[0]
    t = dev(rng.standard_normal((2, 2, 2, 3)))
    e, m = ctx.local_eig(dev(L), dev(W1), dev(W2), dev(R), t, krylov_dim=n)
    assert abs(e - np.linalg.eigvalsh(H)[0]) < 1e-11 * np.abs(H).max()


@pytest.mark.parametrize("m,n", [(1, 1), (1, 6), (6, 1), (8, 8), (12, 40), (64, 64), (130, 70), (96, 200),
                                 (256, 256)])
@pytest.mark.parametrize("absorb", ["right", "left"])
def test_svd_truncate(ctx, pkg, m, n, absorb):
    rng = np.random.default_rng(m * 1000 + n)
    p = min(m, n)
    # graded spectrum so that the weight rule cuts inside it
    M = rng.standard_normal((m, p)) @ np.diag(10.0 ** (-np.arange(p) * 8.0 / max(p, 1))) @ \
        np.linalg.qr(rng.standard_normal((n, p)))[0].T
    chi_max, tol = max(1, (2 * p) // 3), 1e-10
    ab = pkg.ABSORB_RIGHT if absorb == "right" else pkg.ABSORB_LEFT
    res = ctx.svd_truncate(dev(M), chi_max, tol, absorb=ab, normalize=False)
    s_ref = np.linalg.svd(M, compute_uv=False)
    S_gpu = host(res.S)
    assert np.abs(S_gpu - s_ref).max() <= 1e-13 * s_ref[0]
    r_ref = S.truncation_rank(S_gpu, chi_max, tol)
    assert res.rank == r_ref
    Al, Ar = host(res.A_left), host(res.A_right)
    U_r, s_r, Vt_r, _, dw = S.svd_truncate(M, chi_max, tol)
    approx = U_r @ np.diag(s_r[: res.rank]) @ Vt_r if len(s_r) == res.rank else None
    recon = Al @ Ar
    if approx is not None:
        assert np.linalg.norm(recon - approx) <= 1e-12 * np.linalg.norm(M)
    iso = Al if ab == pkg.ABSORB_RIGHT else Ar.T
    assert np.abs(iso.T @ iso - np.eye(res.rank)).max() < 1e-12
    err2 = np.linalg.norm(M - recon) ** 2 / np.sum(s_ref ** 2)
    assert abs(err2 - res.discarded) <= 1e-12 + 1e-9 * res.discarded


def test_svd_normalize_and_rank_deficient(ctx, pkg):
    rng = np.random.default_rng(5)
    M = np.outer(rng.standard_normal(10), rng.standard_normal(6)) * 3.0  # rank 1
    res = ctx.svd_truncate(dev(M), 6, 1e-12, absorb=pkg.ABSORB_RIGHT, normalize=True)
    assert res.rank == 1
    assert abs(np.linalg.norm(host(res.A_right)) - 1.0) < 1e-13
    Z = np.zeros((4, 5))
    res = ctx.svd_truncate(dev(Z), 3, 1e-12)
    assert res.rank == 1 and np.all(host(res.S) == 0.0)


def test_truncation_rank_bit_exact(ctx, pkg):
    rng = np.random.default_rng(0)
    cases = [np.array([1.0, 1e-3, 1e-7]), np.array([1.0, 1.0, 1.0, 0.0]), np.zeros(5),
             np.array([3.0]), np.array([1.0, 0.5, 0.5, 0.5, 1e-9, 1e-9])]
    for _ in range(200):
        n = int(rng.integers(1, 300))
        s = np.sort(np.abs(rng.standard_normal(n)) ** rng.uniform(1, 12))[::-1].copy()
        if rng.random() < 0.3:
            s[rng.integers(0, n):] = s[-1]  # ties
        cases.append(s)
    for s in cases:
        for rule in (pkg.TRUNC_WEIGHT, pkg.TRUNC_RELATIVE):
            for tol, chi in ((1e-12, 10 ** 6), (1e-4, 7), (0.3, 3), (1e-300, 50)):
                mode = S.TRUNC_WEIGHT if rule == pkg.TRUNC_WEIGHT else S.TRUNC_RELATIVE
                assert ctx.truncation_rank(dev(s), chi, tol, rule) == S.truncation_rank(s, chi, tol, mode)


# ---------------------------------------------------------------- sweeps
def _run_sweep(ctx, pkg, W, A0, chi_max, tol, n_sweeps, k, precision, refine=0):
    ch = pkg.Chain(ctx, W, A0, chi_max)
    rep = ctx.sweep(ch, mode=pkg.MODE_EIG, n_sweeps=n_sweeps, refine_sweeps=refine, precision=precision,
                    krylov_dim=k, chi_max=chi_max, tol=tol)
    return rep, [host(t) for t in ch.tensors()]


def test_sweep_c1_tfim_fp64(ctx, pkg):
    """C1: TFIM N=16, g=1, chi_max=32, cutoff 1e-12, 6 sweeps, Krylov 20."""
    n = 16
    W = wl.mpo.tfim(n, 1.0)
    A0 = wl.states.random_mps(n, 2, 32, 0)
    rep, A = _run_sweep(ctx, pkg, W, A0, 32, 1e-12, 6, 20, pkg.FP64)
    e_or, _, log = S.dmrg(W, A0, 32, 1e-12, 6, 20)
    e_ff = X.tfim_free_fermion_energy(n, 1.0)
    assert abs(rep["energy"] - e_or) <= 1e-10 * abs(e_or)
    assert abs(rep["energy"] - e_ff) <= 1e-9 * abs(e_ff)
    assert rep["energy"] >= e_ff - 1e-12 * abs(e_ff)
    assert abs(S.expectation(A, W) - rep["energy"]) <= 1e-10 * abs(e_ff)
    for k in range(1, n):
        assert S.right_isometry_error(A[k]) < 1e-12
    assert abs(np.linalg.norm(A[0]) - 1.0) < 1e-12


def test_sweep_c1_tfim_ed_n14(ctx, pkg):
    n = 14
    W = wl.mpo.tfim(n, 1.0)
    rep, _ = _run_sweep(ctx, pkg, W, wl.states.random_mps(n, 2, 128, 3), 128, 1e-14, 4, 20, pkg.FP64)
    e_ed = X.ground_energy(X.tfim_dense(n, 1.0))
    assert abs(rep["energy"] - e_ed) <= 1e-12 * abs(e_ed) * 10


def test_sweep_mixed_with_refinement(ctx, pkg):
    n = 16
    W = wl.mpo.tfim(n, 1.0)
    A0 = wl.states.random_mps(n, 2, 32, 0)
    rep, _ = _run_sweep(ctx, pkg, W, A0, 32, 1e-12, 4, 20, pkg.BF16X3, refine=1)
    e_or, _, _ = S.dmrg(W, A0, 32, 1e-12, 6, 20)
    assert abs(rep["energy"] - e_or) <= 1e-9 * abs(e_or)


def test_sweep_xxz_reduced_c2(ctx, pkg):
    """C2 shape at a size the oracle finishes quickly: XXZ(1), N=20, chi 48."""
    n, chi = 20, 48
    W = wl.mpo.xxz(n, 1.0)
    A0 = wl.states.random_mps(n, 2, chi, 1)
    rep, A = _run_sweep(ctx, pkg, W, A0, chi, 1e-12, 3, 20, pkg.FP64)
    e_or, A_or, log = S.dmrg(W, A0, chi, 1e-12, 3, 20)
    assert abs(rep["energy"] - e_or) <= 1e-10 * abs(e_or)
    rep2, _ = _run_sweep(ctx, pkg, W, A0, chi, 1e-12, 2, 20, pkg.BF16X3, refine=1)
    assert abs(rep2["energy"] - e_or) <= 1e-9 * abs(e_or)


def test_dmrg_solve_poisson_fp64(ctx, pkg):
    n = 4
    x, h = wl.states.interior_grid(n)
    W = wl.mpo.laplacian_qtt_2d(n, h)
    B = wl.states.poisson_source_mps(n)
    X0 = [b.copy() for b in B]
    X0[0] = 0.1 * X0[0]
    ch = pkg.Chain(ctx, W, X0, 64, B=B)
    rep = ctx.sweep(ch, mode=pkg.MODE_SOLVE, n_sweeps=4, precision=pkg.FP64, chi_max=64, tol=1e-22,
                    pcg_rtol=1e-12, pcg_maxiter=500, precond=pkg.PRECOND_JACOBI)
    u = X.order_b_to_grid(S.mps_to_dense([host(t) for t in ch.tensors()]), n)
    (f1x, f1y), (f2x, f2y) = wl.states.poisson_source_factors(n)
    uref = X.poisson_dst_solve(np.outer(f1x, f1y) + np.outer(f2x, f2y))
    assert np.linalg.norm(u - uref) <= 1e-8 * np.linalg.norm(uref)
    assert rep["local_iters"] > 0


@pytest.mark.parametrize("m,n", [(256, 256), (300, 200), (200, 300), (130, 520)])
@pytest.mark.parametrize("absorb", ["right", "left"])
def test_svd_truncate_fp32_rotations(ctx, pkg, m, n, absorb):
    """The bf16x3 sweep's SVD: FP32 Jacobi rotations, FP64 norms and sums.
    Its accuracy is that of FP32 rotations: singular values within 1e-4 s_0,
    isometries orthonormal within 1e-4."""
    rng = np.random.default_rng(m + 7 * n)
    p = min(m, n)
    M = rng.standard_normal((m, p)) @ np.diag(10.0 ** (-np.arange(p) * 6.0 / p)) @ \
        np.linalg.qr(rng.standard_normal((n, p)))[0].T
    ab = pkg.ABSORB_RIGHT if absorb == "right" else pkg.ABSORB_LEFT
    res = ctx.svd_truncate(dev(M), p // 2, 1e-12, absorb=ab, precision=pkg.BF16X3)
    s_ref = np.linalg.svd(M, compute_uv=False)
    assert np.abs(host(res.S)[:p] - s_ref).max() <= 1e-4 * s_ref[0]
    Al, Ar = host(res.A_left), host(res.A_right)
    iso = Al if ab == pkg.ABSORB_RIGHT else Ar.T
    assert np.abs(iso.T @ iso - np.eye(res.rank)).max() < 1e-4
    err2 = np.linalg.norm(M - Al @ Ar) ** 2 / np.sum(s_ref ** 2)
    assert abs(np.sqrt(err2) - np.sqrt(res.discarded)) <= 1e-4  # norm-wise, FP32 rotations


def test_svd_sweep_counters(ctx, pkg):
    """Per-sweep rotation / visit counters of the mixed split: every count is
    bounded by the p (p - 1) / 2 pairs of a sweep and the visits sum to the
    context's pair-visit counter.  Either the last block sweep rotates
    nothing, or a sweep that rotates at most 1/64 of the pairs hands over to
    the cleanup phase, whose rotations and checked pairs form the last entry."""
    rng = np.random.default_rng(5)
    m = n = 320
    M = rng.standard_normal((m, n)) * (0.9 ** np.arange(n))
    ctx.svd_stats(reset=True)
    ctx.svd_cleanup_stats(reset=True)
    res = ctx.svd_truncate(dev(M), 160, 1e-12, precision=pkg.BF16X3)
    assert res.rank == 160
    st = ctx.svd_stats(reset=True)
    cs = ctx.svd_cleanup_stats(reset=True)
    rot, vis = ctx.svd_sweep_counts()
    print(f"sweep rotations {rot}, cleanup {cs}")
    assert st["calls"] == 1 and len(rot) == len(vis) == st["sweeps"] + 1
    assert rot[0] > 0 and cs["fallbacks"] == 0
    pairs = n * (n - 1) // 2
    assert all(0 <= r <= v <= pairs for r, v in zip(rot, vis))
    assert vis[0] == pairs  # nothing is skipped in the first sweep
    assert sum(vis) == st["pair_visits"]
    if cs["calls"]:
        assert cs["calls"] == 1 and cs["rounds"] >= 1
        assert 0 < rot[-2] <= pairs // 64  # the hand-over condition
    else:
        assert rot[-1] == 0


@pytest.mark.parametrize("m", [1024, 1016, 1020])
def test_svd_cleanup_phase_matches_lapack(ctx, pkg, m):
    """A flat spectrum (a random Gaussian matrix: the slowest case for
    one-sided Jacobi) runs many block sweeps and hands its last ones to the
    cleanup phase.  The result must meet the same bounds as the block sweeps
    alone: singular values within 1e-4 s_0 of LAPACK, an isometric factor
    orthonormal to 1e-4, and M = A_left A_right up to the discarded weight.
    1024 columns form 128 blocks of 8 (the stationary-block schedule, a CTA
    per block pair); 1016 leave the last of 128 blocks empty and 1020 fill it
    half."""
    rng = np.random.default_rng(11)
    n = m
    M = rng.standard_normal((m, n))
    ctx.svd_cleanup_stats(reset=True)
    res = ctx.svd_truncate(dev(M), n, 1e-14, absorb=pkg.ABSORB_RIGHT, normalize=False, precision=pkg.BF16X3)
    cs = ctx.svd_cleanup_stats(reset=True)
    rot, _ = ctx.svd_sweep_counts()
    print(f"flat spectrum {m} x {n}: sweep rotations {rot}, cleanup {cs}")
    assert cs["fallbacks"] == 0
    if m == 1024:
        assert cs["calls"] == 1
    s_ref = np.linalg.svd(M, compute_uv=False)
    assert np.abs(host(res.S) - s_ref).max() <= 1e-4 * s_ref[0]
    Al, Ar = host(res.A_left), host(res.A_right)
    assert np.abs(Al.T @ Al - np.eye(res.rank)).max() < 1e-4
    assert np.linalg.norm(M - Al @ Ar) / np.linalg.norm(M) <= 1e-4


def test_sweep_long_chain_unnormalised_start(ctx, pkg):
    """48 sites from a Gaussian (unnormalised, norm ~1e40) initial MPS: the
    canonicalisation must keep every intermediate inside the FP32 / bf16
    range of the mixed path; the energy reaches the free-fermion value."""
    n, g, chi = 48, 1.3, 32
    W = wl.mpo.tfim(n, g)
    A0 = wl.states.random_mps(n, 2, chi, 9)
    rep, A = _run_sweep(ctx, pkg, W, A0, chi, 1e-12, 3, 20, pkg.BF16X3, refine=1)
    e_ff = X.tfim_free_fermion_energy(n, g)
    assert np.isfinite(rep["energy"])
    assert abs(rep["energy"] - e_ff) <= 1e-9 * abs(e_ff)
    assert all(np.isfinite(a).all() for a in A)
