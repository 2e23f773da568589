"""The learned preconditioner on the GPU: forward and gradient parity with
the oracle, PCG at the Jacobi starting point, and training through the C
call on local systems of the QTT Poisson solve (loss, residual, iterations
against Jacobi-PCG on held-out systems)."""
import numpy as np
import pytest

import workloads as wl
from oracle import mlp as M
from oracle import sweep as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import torch
    assert torch.cuda.is_available()
    import paper_2601_16734_gb300 as pkg
    pkg.build()
    return pkg


@pytest.fixture(scope="module")
def ctx(pkg):
    c = pkg.Context(0, chi_max=64, d=2, D_max=5, krylov_dim=20, chib_max=32)
    yield c
    assert c.device_status() == 0
    c.close()


def dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()


def _spd_system(seed, n=3, i=2):
    """A local system of the 2-D QTT Laplacian (SPD): environments of a
    random mixed-canonical MPS centred on the pair (i, i+1)."""
    x, h = wl.states.interior_grid(n)
    W = wl.mpo.laplacian_qtt_2d(n, h)
    N = 2 * n
    A = S.right_canonicalize(wl.states.random_mps(N, 2, 8, seed))
    for k in range(i):
        chl, d, chr_ = A[k].shape
        Q, Rm = np.linalg.qr(A[k].reshape(chl * d, chr_))
        A[k] = Q.reshape(chl, d, Q.shape[1])
        A[k + 1] = np.einsum("mn,nsc->msc", Rm, A[k + 1])
    L = np.ones((1, 1, 1))
    for k in range(i):
        L = S.left_env(L, A[k], W[k])
    R = np.ones((1, 1, 1))
    for k in range(N - 1, i + 1, -1):
        R = S.right_env(R, A[k], W[k])
    W1, W2 = W[i], W[i + 1]
    H = S.heff_dense(L, W1, W2, R)
    shape = (L.shape[0], 2, 2, R.shape[0])
    b = np.random.default_rng(seed).standard_normal(shape)
    xstar = np.linalg.solve(H, b.reshape(-1)).reshape(shape)
    return L, W1, W2, R, H, b, xstar


def test_forward_and_gradient_match_oracle(ctx, pkg):
    L, W1, W2, R, A, b, xstar = _spd_system(0)
    assert np.linalg.eigvalsh(0.5 * (A + A.T))[0] > 0
    rng = np.random.default_rng(1)
    theta = (rng.standard_normal(M.param_count()) * 0.2).astype(np.float32).astype(np.float64)
    mlp = pkg.Mlp(ctx, theta)
    mlp.set_site(3, 10)
    p, U = mlp.forward(dev(L), dev(W1), dev(W2), dev(R))
    diag = S.heff_diagonal(L, W1, W2, R)
    X = M.features(diag, L, R, 3, 10)
    o, _ = M.forward(theta, X)
    p_ref, U_ref = M.precond_factors(o, diag)
    assert np.abs(p.cpu().numpy() - p_ref).max() <= 1e-5 * np.abs(p_ref).max()
    assert np.abs(U.cpu().numpy() - U_ref).max() <= 1e-5 * max(np.abs(U_ref).max(), 1e-3)
    Aop = lambda v: S.heff_apply(L, W1, W2, R, v)
    loss_ref, g_ref = M.loss_and_grad(theta, X, diag, b, xstar, Aop)
    mlp.zero_grad()
    mlp.loss_grad(dev(L), dev(W1), dev(W2), dev(R), dev(b), dev(xstar))
    g = mlp.grad.cpu().numpy().astype(np.float64)
    assert abs(mlp.loss.item() - loss_ref) <= 1e-5 * max(1.0, loss_ref)
    assert np.linalg.norm(g - g_ref) <= 1e-4 * np.linalg.norm(g_ref)
    mlp.close()


def test_adam_step_matches_oracle(ctx, pkg):
    L, W1, W2, R, A, b, xstar = _spd_system(2)
    rng = np.random.default_rng(3)
    theta = (rng.standard_normal(M.param_count()) * 0.2).astype(np.float32).astype(np.float64)
    mlp = pkg.Mlp(ctx, theta)
    mlp.zero_grad()
    mlp.loss_grad(dev(L), dev(W1), dev(W2), dev(R), dev(b), dev(xstar))
    g = mlp.grad.cpu().numpy().astype(np.float64)
    mlp.adam_step(1e-3)
    ref = M.adam_step(theta.copy(), g, np.zeros_like(g), np.zeros_like(g), 1, 1e-3)
    assert np.abs(mlp.params.cpu().numpy() - ref).max() < 1e-6
    mlp.close()


def _poisson_systems(pkg, ctx, n, seeds, chi):
    from paper_2601_16734_gb300 import precond_train as PT
    x, h = wl.states.interior_grid(n)
    W = wl.mpo.laplacian_qtt_2d(n, h)
    out = []
    for sd in seeds:
        B = wl.states.separable_qtt_2d(wl.states.random_poisson_source_terms(n, sd), n)
        X0 = [bb.copy() for bb in B]
        X0[0] = 0.1 * X0[0]
        out += PT.collect_local_systems(ctx, W, B, X0, chi, sweeps=2)
    return out


def test_pcg_at_init_is_jacobi(ctx, pkg):
    from paper_2601_16734_gb300 import precond_train as PT
    systems = _poisson_systems(pkg, ctx, 4, [100], 16)
    mlp = pkg.Mlp(ctx, M.init_params(7))
    it_j, res_j = PT.pcg_iterations(ctx, systems, pkg.PRECOND_JACOBI)
    it_m, res_m = PT.pcg_iterations(ctx, systems, pkg.PRECOND_MLP, mlp=mlp)
    assert res_j <= 1e-10 and res_m <= 1e-10
    assert abs(it_m - it_j) <= len(systems)  # FP32 softplus(1) rounding only
    mlp.close()


def test_training_lowers_the_loss_and_keeps_the_residual(ctx, pkg):
    """Train on the local systems of 6 random-source solves (one seemps_mlp_train
    call), evaluate on 2 held-out solves: the training loss falls, PCG with the
    trained network reaches the same relative residual as Jacobi, and the
    iteration counts are reported.  The diagonal-plus-rank-4 form does not cut
    iterations on these systems (even the exact four lowest eigenvectors as a
    coarse space remove only ~20 % of them), so no gain is asserted; the
    bound below only guards against a broken preconditioner."""
    from paper_2601_16734_gb300 import precond_train as PT
    train = _poisson_systems(pkg, ctx, 5, range(100, 106), 32)
    test = _poisson_systems(pkg, ctx, 5, range(200, 202), 32)
    mlp = pkg.Mlp(ctx, M.init_params(11))
    hist = PT.train(mlp, train, steps=300, lr=3e-3, batch=16, log_every=100, log=lambda s: None)
    it_j, res_j = PT.pcg_iterations(ctx, test, pkg.PRECOND_JACOBI)
    it_m, res_m = PT.pcg_iterations(ctx, test, pkg.PRECOND_MLP, mlp=mlp)
    print(f"held-out PCG iterations: Jacobi {it_j}, learned {it_m} (ratio {it_m / it_j:.3f}); "
          f"train loss {hist[0][1]:.3e} -> {hist[-1][1]:.3e}")
    assert res_j <= 1e-10 and res_m <= 1e-10
    assert hist[-1][1] < hist[0][1]
    assert it_m <= 2 * it_j
    mlp.close()
