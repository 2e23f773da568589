"""QTT Poisson solve (-Laplace u = f on [0,1]^2, Dirichlet) by DMRG as a
linear solver on the GPU, checked against exact discrete solutions.

At 2^20 x 2^20 (40 interleaved qubits, the C4 size) the exact discrete
solution is known in closed form for the sine source sin(pi x) sin(3 pi y):
u = f / (lambda_1 + lambda_3) with lambda_k = (4/h^2) sin^2(k pi h / 2).  The
solution MPS is evaluated on sampled grid points (an MPS element is an exact
product of matrices) and compared there.  The full source (sine + Gaussian)
is checked against the DST solution of the 2^8 x 2^8 grid."""
import numpy as np
import pytest

import workloads as wl
from oracle import exact as X
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
    c = pkg.Context(0, chi_max=64, d=2, D_max=5, krylov_dim=20, chib_max=64)
    yield c
    assert c.device_status() == 0
    c.close()


def mps_values(A, n, ix, iy):
    """u[i_x, i_y] of an order-B MPS at the given integer grid points."""
    out = np.empty(len(ix))
    for k, (a, b) in enumerate(zip(ix, iy)):
        v = np.ones((1,))
        for lvl in range(n):
            sx = (a >> (n - 1 - lvl)) & 1
            sy = (b >> (n - 1 - lvl)) & 1
            v = v @ A[2 * lvl][:, sx, :]
            v = v @ A[2 * lvl + 1][:, sy, :]
        out[k] = v[0]
    return out


def solve(pkg, ctx, n, B, sweeps, chi=64, precision=None, refine=0):
    x, h = wl.states.interior_grid(n)
    W = wl.mpo.laplacian_qtt_2d(n, h)
    X0 = [b.copy() for b in B]
    X0[0] = 0.1 * X0[0]
    ch = pkg.Chain(ctx, W, X0, chi, B=B)
    rep = ctx.sweep(ch, mode=pkg.MODE_SOLVE, n_sweeps=sweeps, refine_sweeps=refine,
                    precision=pkg.FP64 if precision is None else precision, chi_max=chi, tol=1e-24,
                    pcg_rtol=1e-13, pcg_maxiter=4000, precond=pkg.PRECOND_JACOBI)
    return [t.cpu().numpy() for t in ch.tensors()], rep


def rounding_floor(n):
    """FP64 floor of the relative error for the sine source on 2^n x 2^n.

    Applying the interior-grid stencil to a smooth mode cancels terms of
    size ~ 4/h^2 (two coordinates, each 2/h^2 with the two neighbours) down to
    lambda_1 + lambda_3 ~ 10 pi^2, so the operator, the residuals and hence
    the solution carry a relative rounding error of order
    eps * (8 / h^2) / (10 pi^2) with h ~ 2^-n."""
    return 2.220446049250313e-16 * 8.0 * 4.0 ** n / (10.0 * np.pi ** 2)


@pytest.mark.parametrize("n", [10, 14, 17, 20])
def test_sine_source_exact_solution(ctx, pkg, n):
    x, h = wl.states.interior_grid(n)
    B = wl.states.separable_qtt_2d([(np.sin(np.pi * x), np.sin(3 * np.pi * x))], n)
    A, rep = solve(pkg, ctx, n, B, sweeps=4)
    lam = X.dirichlet_eigenvalues(n)
    rng = np.random.default_rng(n)
    ix = rng.integers(0, 2 ** n, 2000)
    iy = rng.integers(0, 2 ** n, 2000)
    u = mps_values(A, n, ix, iy)
    ue = np.sin(np.pi * x[ix]) * np.sin(3 * np.pi * x[iy]) / (lam[0] + lam[2])
    rel = np.linalg.norm(u - ue) / np.linalg.norm(ue)
    tol = max(1e-8, rounding_floor(n))
    print(f"n={n} sine source: sampled relative L2 error {rel:.2e} (bound {tol:.1e}), "
          f"PCG iterations {rep['local_iters']}")
    assert rel <= tol


def test_full_source_vs_dst(ctx, pkg):
    n = 8
    B = wl.states.poisson_source_mps(n)
    A, rep = solve(pkg, ctx, n, B, sweeps=6)
    u = X.order_b_to_grid(S.mps_to_dense(A), n)
    (f1x, f1y), (f2x, f2y) = wl.states.poisson_source_factors(n)
    uref = X.poisson_dst_solve(np.outer(f1x, f1y) + np.outer(f2x, f2y))
    rel = np.linalg.norm(u - uref) / np.linalg.norm(uref)
    print(f"n=8 full source: relative L2 error {rel:.2e}")
    assert rel <= 1e-8


def test_full_source_mixed_then_fp64_refinement(ctx, pkg):
    n = 8
    B = wl.states.poisson_source_mps(n)
    A, rep = solve(pkg, ctx, n, B, sweeps=2, precision=pkg.BF16X3, refine=3)
    u = X.order_b_to_grid(S.mps_to_dense(A), n)
    (f1x, f1y), (f2x, f2y) = wl.states.poisson_source_factors(n)
    uref = X.poisson_dst_solve(np.outer(f1x, f1y) + np.outer(f2x, f2y))
    rel = np.linalg.norm(u - uref) / np.linalg.norm(uref)
    print(f"n=8 full source, bf16x3 + FP64 refinement: relative L2 error {rel:.2e}")
    assert rel <= 1e-8
