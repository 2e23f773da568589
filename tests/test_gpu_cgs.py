"""Global conjugate gradients on MPS (Sect. 3.2.1; seemps_cgs_solve) vs the
oracle's cgs_solve and the dense system:

- with a bond dimension that holds every vector exactly, the iterates are
  textbook CG on the dense system and the oracle's, step by step;
- run to convergence it solves U x = b (numpy.linalg.solve);
- with truncation (bond 6 on 10 sites) the residual history follows the
  oracle's step by step (FP64, same compressions);
- bf16x3 sweeps reach their floor (2e-3 here), FP64 steps from there 1e-9;
- a guess bond above chi_max and an indefinite U are refused as status codes.
U = shift I + tridiag(-1, 2, -1) as a QTT MPO (D = 3).
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


def _shifted_laplacian(n, shift):
    W = wl.mpo.laplacian_qtt_1d(n, 1.0)
    W[-1] = W[-1].copy()
    W[-1][0, :, :, 0] += shift * np.eye(2)
    return W


def _dense(A):
    return S.mps_to_dense(A).reshape(-1)


def _solve(pkg, W, b, x0, chi, **kw):
    chib = max(t.shape[2] for t in b)
    ctx = pkg.Context(0, chi_max=chi, d=2, D_max=3, krylov_dim=2, chib_max=chi + max(chi, chib))
    try:
        x, rep = ctx.cgs_solve(W, b, x0, chi, **kw)
        x = [t.detach().cpu().numpy() for t in x]
        assert ctx.device_status() == 0
    finally:
        ctx.close()
    return x, rep


def test_iterates_are_textbook_cg(pkg):
    n = 6
    W = _shifted_laplacian(n, 0.5)
    U = S.mpo_to_dense(W)
    b = wl.states.random_mps(n, 2, 4, 4)
    x0 = wl.states.random_mps(n, 2, 3, 5)
    for steps in (1, 2, 3):
        x, rep = _solve(pkg, W, b, x0, 8, tol=1e-30, rtol=0.0, maxiter=steps)
        assert rep["iterations"] == steps
        xo, _, _, _ = S.cgs_solve(W, b, x0, 8, 1e-30, 0.0, steps)
        assert np.linalg.norm(_dense(x) - _dense(xo)) <= 1e-10 * np.linalg.norm(_dense(xo))
        # textbook CG on the dense system
        xd = _dense(x0).copy()
        r = _dense(b) - U @ xd
        p = r.copy()
        for _ in range(steps):
            a = (r @ r) / (p @ U @ p)
            xd = xd + a * p
            rn = _dense(b) - U @ xd
            p = rn + (rn @ rn) / (r @ r) * p
            r = rn
        assert np.linalg.norm(_dense(x) - xd) <= 1e-10 * np.linalg.norm(xd)


def test_converges_to_the_solution(pkg):
    n = 6
    W = _shifted_laplacian(n, 0.5)
    b = wl.states.random_mps(n, 2, 4, 6)
    x, rep = _solve(pkg, W, b, wl.states.random_mps(n, 2, 2, 7), 8, tol=1e-30, rtol=1e-10, maxiter=100)
    assert rep["residual"] < 1e-10 * rep["norm_b"]
    assert abs(rep["norm_b"] - np.linalg.norm(_dense(b))) <= 1e-12 * rep["norm_b"]
    ref = np.linalg.solve(S.mpo_to_dense(W), _dense(b))
    assert np.linalg.norm(_dense(x) - ref) <= 1e-9 * np.linalg.norm(ref)
    _, res_o, k_o, _ = S.cgs_solve(W, b, wl.states.random_mps(n, 2, 2, 7), 8, 1e-30, 1e-10, 100)
    assert abs(rep["iterations"] - k_o) <= 1


def test_truncated_follows_the_oracle(pkg):
    """Bond 6 on 10 sites (1024 unknowns): every compression truncates."""
    n, chi, steps = 10, 6, 6
    W = _shifted_laplacian(n, 0.3)
    b = wl.states.random_mps(n, 2, 5, 8)
    x0 = wl.states.random_mps(n, 2, 4, 9)
    x, rep = _solve(pkg, W, b, x0, chi, tol=1e-30, rtol=0.0, maxiter=steps)
    xo, res_o, k_o, hist_o = S.cgs_solve(W, b, x0, chi, 1e-30, 0.0, steps)
    assert rep["iterations"] == k_o == steps
    h = np.array(rep["residual_history"])
    assert np.abs(h - np.array(hist_o)).max() <= 1e-8 * hist_o[0]
    assert max(t.shape[2] for t in x) <= chi
    assert np.linalg.norm(_dense(x) - _dense(xo)) <= 1e-8 * np.linalg.norm(_dense(xo))


def test_mixed_then_fp64_refinement(pkg):
    """bf16x3 sweeps carry a relative error near 2^-16 per product into every
    compression, which CG (condition number 9 here) turns into a residual
    floor near 1e-3: the mixed run reaches 2e-3; FP64 steps started from its
    x then reach 1e-9 and the dense solution."""
    n, chi = 10, 32
    W = _shifted_laplacian(n, 0.5)
    b = wl.states.random_mps(n, 2, 8, 10)
    x, rep = _solve(pkg, W, b, wl.states.random_mps(n, 2, 4, 11), chi, tol=1e-14, rtol=2e-3, maxiter=60,
                    precision=pkg.BF16X3)
    assert rep["residual"] < 2e-3 * rep["norm_b"]
    x2, rep2 = _solve(pkg, W, b, x, chi, tol=1e-30, rtol=1e-9, maxiter=60, precision=pkg.FP64)
    assert rep2["residual"] < 1e-9 * rep2["norm_b"]
    ref = np.linalg.solve(S.mpo_to_dense(W), _dense(b))
    assert np.linalg.norm(_dense(x2) - ref) <= 1e-8 * np.linalg.norm(ref)


def test_refused_inputs(pkg):
    from paper_2601_16734_gb300 import abi
    n = 6
    W = _shifted_laplacian(n, 0.5)
    b = wl.states.random_mps(n, 2, 4, 12)
    with pytest.raises(abi.SeempsError) as e:  # guess bond 8 > chi_max 4
        _solve(pkg, W, b, wl.states.random_mps(n, 2, 8, 13), 4, maxiter=3)
    assert e.value.status == 1
    Wneg = [w.copy() for w in W]
    Wneg[0] = -Wneg[0]  # U -> -U, negative definite
    with pytest.raises(abi.SeempsError) as e:
        _solve(pkg, Wneg, b, wl.states.random_mps(n, 2, 2, 14), 8, maxiter=3)
    assert e.value.status == 1
