"""QTT Poisson solve (-Laplace u = f on [0,1]^2, Dirichlet) by DMRG as a
linear solver on the GPU, checked against exact discrete solutions.

At 2^20 x 2^20 (40 interleaved qubits, the C4 size) the exact discrete
solution is known in closed form for the sine source sin(pi x) sin(3 pi y):
u = f / (lambda_1 + lambda_3) with lambda_k = (4/h^2) sin^2(k pi h / 2); for
the full source (sine + Gaussian, both separable) it is the eigen-expansion
of the stencil (oracle.exact.poisson_separable_solution).  The solution MPS
is evaluated on sampled grid points (an MPS element is an exact product of
matrices) and compared there.

FP64 environments of the QTT Laplacian bound the relative error near
eps 4^n / 40 (the CPU oracle shows the same: 3e-10 at n = 14, 5e-8 at
n = 17, 3e-6 at n = 20), so the FP64 runs stop at n = 14 and the large
sizes run with double-FP64 environments (FP64X2), all against 1e-8."""
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
    # the C4 source's TT-SVD at 2^20 points has bonds up to 153
    c = pkg.Context(0, chi_max=64, d=2, D_max=5, krylov_dim=20, chib_max=160)
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


def solve(pkg, ctx, n, B, sweeps, chi=64, precision=None, refine=0, maxiter=4000):
    x, h = wl.states.interior_grid(n)
    W = wl.mpo.laplacian_qtt_2d(n, h)
    X0 = [b.copy() for b in B]
    X0[0] = 0.1 * X0[0]
    ch = pkg.Chain(ctx, W, X0, chi, B=B, extended=precision == pkg.FP64X2)
    rep = ctx.sweep(ch, mode=pkg.MODE_SOLVE, n_sweeps=sweeps, refine_sweeps=refine,
                    precision=pkg.FP64 if precision is None else precision, chi_max=chi, tol=1e-24,
                    pcg_rtol=1e-13, pcg_maxiter=maxiter, precond=pkg.PRECOND_JACOBI)
    return [t.cpu().numpy() for t in ch.tensors()], rep


def sine_error(pkg, ctx, n, precision, sweeps=4):
    x, h = wl.states.interior_grid(n)
    B = wl.states.separable_qtt_2d([(np.sin(np.pi * x), np.sin(3 * np.pi * x))], n)
    A, rep = solve(pkg, ctx, n, B, sweeps=sweeps, precision=precision)
    lam = X.dirichlet_eigenvalues(n)
    rng = np.random.default_rng(n)
    ix = rng.integers(0, 2 ** n, 2000)
    iy = rng.integers(0, 2 ** n, 2000)
    u = mps_values(A, n, ix, iy)
    ue = np.sin(np.pi * x[ix]) * np.sin(3 * np.pi * x[iy]) / (lam[0] + lam[2])
    return np.linalg.norm(u - ue) / np.linalg.norm(ue), rep


@pytest.mark.parametrize("n", [10, 14])
def test_sine_source_exact_solution_fp64(ctx, pkg, n):
    rel, rep = sine_error(pkg, ctx, n, pkg.FP64)
    print(f"n={n} sine source, FP64: sampled relative L2 error {rel:.2e}, PCG iterations {rep['local_iters']}")
    assert rel <= 1e-8


@pytest.mark.parametrize("n", [14, 17, 20])
def test_sine_source_exact_solution_fp64x2(ctx, pkg, n):
    rel, rep = sine_error(pkg, ctx, n, pkg.FP64X2)
    print(f"n={n} sine source, FP64X2: sampled relative L2 error {rel:.2e}, PCG iterations {rep['local_iters']}")
    assert rel <= 1e-8


def test_full_source_n20_fp64x2(ctx, pkg):
    """The C4 source at 2^20 x 2^20: sine plus the Gaussian of sigma 0.05 at
    (0.3, 0.6), against the stencil's eigen-expansion at sampled points."""
    n = 20
    B = wl.states.poisson_source_mps(n)
    # the chi = 64 local systems are very ill-conditioned: Jacobi-PCG is capped at
    # 2000 iterations per pair and the sweeps carry the solve the rest of the way
    A, rep = solve(pkg, ctx, n, B, sweeps=3, precision=pkg.FP64X2, maxiter=2000)
    rng = np.random.default_rng(7)
    ix = rng.integers(0, 2 ** n, 2000)
    iy = rng.integers(0, 2 ** n, 2000)
    u = mps_values(A, n, ix, iy)
    ue = X.poisson_separable_solution(n, list(wl.states.poisson_source_factors(n)), ix, iy, modes=1024)
    rel = np.linalg.norm(u - ue) / np.linalg.norm(ue)
    print(f"n=20 full source, FP64X2: sampled relative L2 error {rel:.2e}, PCG iterations {rep['local_iters']}, "
          f"max bond {max(t.shape[2] for t in A)}")
    assert rel <= 1e-8


@pytest.mark.skipif(np.finfo(np.longdouble).eps > 1e-18, reason="long double is not wider than FP64 here")
def test_fp64x2_solve_matches_extended_oracle(ctx, pkg):
    """Same inputs, same sweeps: the GPU's double-FP64 solve and the oracle's
    extended-precision solve give the same solution vector.  (A small grid:
    on aarch64 numpy's long double is software binary128.)"""
    n = 5
    x, h = wl.states.interior_grid(n)
    W = wl.mpo.laplacian_qtt_2d(n, h)
    B = wl.states.poisson_source_mps(n)
    X0 = [b.copy() for b in B]
    X0[0] = 0.1 * X0[0]
    A, _ = solve(pkg, ctx, n, B, sweeps=2, precision=pkg.FP64X2)
    Ao, _ = S.dmrg_solve(W, B, X0, 64, 1e-24, 2, pcg_rtol=1e-13, pcg_maxiter=4000, extended=True)
    u, uo = S.mps_to_dense(A), S.mps_to_dense(Ao)
    rel = np.linalg.norm(u - uo) / np.linalg.norm(uo)
    print(f"n=5 full source: GPU FP64X2 vs oracle extended {rel:.2e}")
    assert rel <= 1e-10


def _pair_environments(n, i):
    """Laplacian MPO, the exact sine solution as a mixed-canonical MPS with the
    centre on (i, i+1), and long-double environments L_i, R_{i+2}."""
    x, h = wl.states.interior_grid(n)
    W = wl.mpo.laplacian_qtt_2d(n, h)
    A = S.right_canonicalize(wl.states.separable_qtt_2d([(np.sin(np.pi * x), np.sin(3 * np.pi * x))], n))
    for k in range(i):
        chl, d, chr_ = A[k].shape
        Q, Rm = np.linalg.qr(A[k].reshape(chl * d, chr_))
        A[k] = Q.reshape(chl, d, Q.shape[1])
        A[k + 1] = np.einsum("mn,nsc->msc", Rm, A[k + 1])
    Lenv = np.ones((1, 1, 1), dtype=np.longdouble)
    for k in range(i):
        Lenv = S.left_env(Lenv, A[k], W[k])
    Renv = np.ones((1, 1, 1), dtype=np.longdouble)
    for k in range(2 * n - 1, i + 1, -1):
        Renv = S.right_env(Renv, A[k], W[k])
    return W, A, Lenv, Renv


def _dd(t, dev):
    """Long-double array -> double-FP64 device tensor (hi parts, then lo parts)."""
    import torch
    hi = t.astype(np.float64)
    lo = (t - hi.astype(np.longdouble)).astype(np.float64)
    return torch.from_numpy(np.ascontiguousarray(np.stack([hi, lo]))).to(dev)


@pytest.mark.skipif(np.finfo(np.longdouble).eps > 1e-18, reason="long double is not wider than FP64 here")
def test_fp64x2_heff_and_env_update_vs_long_double(ctx, pkg):
    """Element-wise parity of the double-FP64 entry points on the Laplacian's
    cancelling channels: H_n theta rounded once to FP64, and the environment
    update carried to ~1e-17 of its largest entry (FP64 leaves ~1e-16)."""
    import torch
    n, i = 8, 7
    W, A, Lenv, Renv = _pair_environments(n, i)
    dev = ctx.device
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(dev)
    theta = S.two_site(A[i], A[i + 1])
    yref = S.heff_apply(Lenv, W[i], W[i + 1], Renv, theta)
    y = ctx.heff_apply(_dd(Lenv, dev), t(W[i]), t(W[i + 1]), _dd(Renv, dev), t(theta), precision=pkg.FP64X2)
    err = np.abs(y.cpu().numpy().astype(np.longdouble) - yref).max() / np.abs(yref).max()
    print(f"FP64X2 heff_apply: max error {float(err):.2e} of max |y|")
    assert err <= 2e-15
    # left environment across site i
    Lref = S.left_env(Lenv, A[i], W[i])
    Lout = ctx.env_update(pkg.LEFT, _dd(Lenv, dev), t(A[i]), t(W[i]), precision=pkg.FP64X2)
    got = Lout[0].cpu().numpy().astype(np.longdouble) + Lout[1].cpu().numpy().astype(np.longdouble)
    err = np.abs(got - Lref).max() / np.abs(Lref).max()
    print(f"FP64X2 env_update: max error {float(err):.2e} of max |L|")
    assert err <= 1e-17


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
