"""Two-site TDVP in imaginary time (Sect. 7.3, TDVP; generator L = -H) on the
GPU against the oracle:

- the one-site effective operator (seemps_heff1_apply) element by element;
- the Krylov exponential (seemps_local_expm) against the oracle's Krylov
  exponential on the same start vector, and against scipy's expm when the
  Krylov space is the whole local space;
- the TDVP sweep (seemps_sweep, TDVP mode) against exp(-t H) psi at the full
  bond dimension, against the oracle's TDVP with truncation, and, after a
  long imaginary time, against the exact ground energy.
"""
import numpy as np
import pytest
import scipy.linalg

import workloads as wl
from oracle import exact as X
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
    c = pkg.Context(0, chi_max=160, d=3, D_max=5, krylov_dim=24)
    yield c
    assert c.device_status() == 0
    c.close()


def dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def relerr(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def close(a, b, tol):
    """Norm-wise and element-wise (largest error over the largest entry) within tol."""
    assert relerr(a, b) < tol, relerr(a, b)
    assert np.abs(a - b).max() <= tol * max(np.abs(b).max(), 1e-300), np.abs(a - b).max() / np.abs(b).max()


def _dense(A):
    v = S.mps_to_dense(A).reshape(-1)
    return v / np.linalg.norm(v)


def _site_problem(chil, chir, D_l, D_r, d, seed):
    rng = np.random.default_rng(seed)
    L = rng.standard_normal((chil, D_l, chil))
    R = rng.standard_normal((chir, D_r, chir))
    L = 0.5 * (L + L.transpose(2, 1, 0))  # symmetric environments: a symmetric operator
    R = 0.5 * (R + R.transpose(2, 1, 0))
    W = rng.standard_normal((D_l, d, d, D_r))
    W = 0.5 * (W + W.transpose(0, 2, 1, 3))
    A = rng.standard_normal((chil, d, chir))
    return L, W, R, A


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
@pytest.mark.parametrize("shape", [(1, 4, 1, 5, 2), (7, 9, 3, 4, 2), (70, 129, 5, 5, 2), (33, 40, 4, 3, 3)])
def test_heff1_apply_matches_oracle(ctx, pkg, prec, shape):
    chil, chir, D_l, D_r, d = shape
    L, W, R, A = _site_problem(chil, chir, D_l, D_r, d, sum(shape))
    p = pkg.FP64 if prec == "fp64" else pkg.BF16X3
    y = host(ctx.heff1_apply(dev(L), dev(W), dev(R), dev(A), precision=p))
    ref = S.heff1_apply(L, W, R, A)
    close(y, ref, (1e-12 if prec == "fp64" else 2e-4))  # bf16x3: about 2^-16 per product


@pytest.mark.parametrize("tau", [-0.25, 0.25])
def test_local_expm_two_site_matches_oracle(ctx, pkg, tau):
    """Krylov dimension 12 below the local dimension 5 * 2 * 2 * 5 = 100: the
    same Krylov approximation on both sides."""
    n = 8
    W = wl.mpo.xxz(n, 0.8)
    A = S.right_canonicalize(wl.states.random_mps(n, 2, 5, 9))
    Lenv = np.ones((1, 1, 1))
    for i in range(3):
        Lenv = S.left_env(Lenv, A[i], W[i])
    Renv = np.ones((1, 1, 1))
    for i in range(n - 1, 4, -1):
        Renv = S.right_env(Renv, A[i], W[i])
    th = S.two_site(A[3], A[4])
    mv = lambda v: S.heff_apply(Lenv, W[3], W[4], Renv, v)  # noqa: E731
    x, m, a0 = S.krylov_expm(mv, th, tau, 12)
    t = dev(th)
    e, it = ctx.local_expm(dev(Lenv), dev(W[3]), dev(W[4]), dev(Renv), t, tau, krylov_dim=12)
    assert it == m == 12
    assert abs(e - a0) <= 1e-12 * abs(a0)
    assert relerr(host(t), x / np.linalg.norm(x)) < 1e-11


def test_local_expm_mixed_close_to_oracle(ctx, pkg):
    """bf16x3 operator products and an FP32 Krylov basis: the normalised
    result within 1e-4 of the oracle's (the products' relative error is near
    2^-16; |tau| ||H|| is O(1) here)."""
    L, W, R, A = _site_problem(60, 75, 4, 4, 2, 23)
    mv = lambda v: S.heff1_apply(L, W, R, v)  # noqa: E731
    nrm = np.linalg.norm(mv(A)) / np.linalg.norm(A)
    tau = -0.5 / nrm
    x, m, a0 = S.krylov_expm(mv, A, tau, 16)
    t = dev(A)
    e, it = ctx.local_expm(dev(L), dev(W), None, dev(R), t, tau, krylov_dim=16, precision=pkg.BF16X3)
    assert it == m == 16
    assert abs(e - a0) <= 1e-4 * nrm
    assert relerr(host(t), x / np.linalg.norm(x)) < 1e-4


def test_local_expm_one_site_full_space_is_exact(ctx, pkg):
    """One-site operator of local dimension 3 * 2 * 4 = 24 with Krylov
    dimension 24: the Krylov space is the whole space, the result the exact
    normalised exp(tau H) a."""
    L, W, R, A = _site_problem(3, 4, 3, 2, 2, 17)
    H = np.stack([S.heff1_apply(L, W, R, e.reshape(A.shape)).reshape(-1)
                  for e in np.eye(A.size)], axis=1)
    for tau in (-0.3, 0.15):
        ref = scipy.linalg.expm(tau * H) @ A.reshape(-1)
        ref /= np.linalg.norm(ref)
        t = dev(A)
        _, it = ctx.local_expm(dev(L), dev(W), None, dev(R), t, tau, krylov_dim=24)
        assert it <= 24
        assert relerr(host(t).reshape(-1), ref) < 1e-11


def _tdvp(ctx, pkg, W, A0, chi, dt, steps, precision=None, refine=0, krylov=20):
    ch = pkg.Chain(ctx, W, A0, chi)
    rep = ctx.sweep(ch, mode=pkg.MODE_TDVP, n_sweeps=steps, refine_sweeps=refine,
                    precision=pkg.FP64 if precision is None else precision, krylov_dim=krylov, chi_max=chi,
                    tol=1e-30, tdvp_dt=dt)
    return rep, [host(t) for t in ch.tensors()]


def test_tdvp_exact_at_full_bond_dimension(ctx, pkg):
    n = 6
    W = wl.mpo.tfim(n, 1.1)
    A0 = wl.states.random_mps(n, 2, 8, 5)
    H = S.mpo_to_dense(W)
    for dt, steps in ((0.1, 4), (0.35, 2)):
        ref = scipy.linalg.expm(-dt * steps * H) @ _dense(A0)
        ref /= np.linalg.norm(ref)
        _, A = _tdvp(ctx, pkg, W, A0, 8, dt, steps)
        v = _dense(A)
        assert np.linalg.norm(v - np.sign(v @ ref) * ref) <= 1e-10


def test_tdvp_truncated_matches_oracle(ctx, pkg):
    """Bond 6 on 10 sites of XXZ: every split truncates; the GPU sweep and the
    oracle's TDVP take the same steps."""
    n, chi, dt, steps = 10, 6, 0.2, 3
    W = wl.mpo.xxz(n, 0.6)
    A0 = wl.states.random_mps(n, 2, chi, 13)
    rep, A = _tdvp(ctx, pkg, W, A0, chi, dt, steps)
    E_or, Ao, log = S.tdvp(W, A0, dt, steps, chi, 1e-30, 20)
    assert max(a.shape[2] for a in A) == chi
    assert log.error > 1e-8
    v, vo = _dense(A), _dense(Ao)
    assert np.linalg.norm(v - np.sign(v @ vo) * vo) <= 1e-9
    E = S.expectation(A, W) / S.overlap(A, A)
    assert abs(E - E_or) <= 1e-10 * abs(E_or)
    assert abs(rep["error_bound"] - log.error) <= 1e-6 * log.error


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_tdvp_imaginary_time_ground_state(ctx, pkg, prec):
    """TFIM g = 1.5 (gapped), 16 sites, bond 16, t = 20: the ground energy of
    the free-fermion solution to 1e-9 (the mixed run ends with 10 FP64
    steps)."""
    n, g = 16, 1.5
    W = wl.mpo.tfim(n, g)
    A0 = wl.states.random_mps(n, 2, 16, 21)
    if prec == "fp64":
        rep, A = _tdvp(ctx, pkg, W, A0, 16, 0.5, 40)
    else:
        rep, A = _tdvp(ctx, pkg, W, A0, 16, 0.5, 30, precision=pkg.BF16X3, refine=10)
    e_ff = X.tfim_free_fermion_energy(n, g)
    E = S.expectation(A, W) / S.overlap(A, A)
    assert abs(E - e_ff) <= 1e-9 * abs(e_ff)
    assert abs(rep["energy"] - e_ff) <= 1e-8 * abs(e_ff)
    assert rep["half_sweeps"] == 80


def test_tdvp_rejects_bad_time_step(ctx, pkg):
    from paper_2601_16734_gb300 import abi
    n = 4
    ch = pkg.Chain(ctx, wl.mpo.tfim(n, 1.0), wl.states.random_mps(n, 2, 4, 1), 4)
    for dt in (0.0, -0.1, float("nan")):
        with pytest.raises(abi.SeempsError) as e:
            ctx.sweep(ch, mode=pkg.MODE_TDVP, chi_max=4, tdvp_dt=dt)
        assert e.value.status == 1
    assert ctx.device_status() == 0
