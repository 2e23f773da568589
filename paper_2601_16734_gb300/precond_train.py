"""Training of the learned local preconditioner on the GPU.

Local systems H_n x = b_n are collected from DMRG-as-solver runs (Sect.
3.2.3) driven through the library: after Jacobi-PCG sweeps have converged,
the walk over the pairs snapshots each pair's environments, its right-hand
side b_n and the exact local solution x* (PCG to a tight tolerance).  The
network is then trained with the library's own forward/backward and Adam
kernels on the loss |x* - P b|_A^2 / (x*^T b).
"""
from __future__ import annotations

from dataclasses import dataclass

import torch

from . import abi


@dataclass
class LocalSystem:
    L: torch.Tensor
    W1: torch.Tensor
    W2: torch.Tensor
    R: torch.Tensor
    b: torch.Tensor
    xstar: torch.Tensor
    x0: torch.Tensor
    site: int
    n_sites: int


def collect_local_systems(ctx: abi.Context, W: list, B: list, X0: list, chi_max: int, sweeps: int = 2,
                          tol: float = 1e-14, pcg_rtol: float = 1e-12, solve_rtol: float = 1e-13) -> list:
    """Run DMRG-solve sweeps (Jacobi-PCG) and snapshot every pair's local system."""
    chain = abi.Chain(ctx, W, X0, chi_max, B=B)
    kw = dict(mode=abi.MODE_SOLVE, precision=abi.FP64, chi_max=chi_max, tol=tol, pcg_rtol=pcg_rtol,
              precond=abi.PRECOND_JACOBI)
    ctx.sweep(chain, n_sweeps=sweeps, **kw)
    N, D, d = chain.N, chain.Dlist, chain.d
    out = []
    for i in range(N - 1):
        chl, chm, chr_ = chain.chi[i], chain.chi[i + 1], chain.chi[i + 2]
        bl, bm, br = chain.chib[i], chain.chib[i + 1], chain.chib[i + 2]
        L = chain.L[i][: chl * D[i] * chl].view(chl, D[i], chl).clone()
        R = chain.R[i + 2][: chr_ * D[i + 2] * chr_].view(chr_, D[i + 2], chr_).clone()
        F = chain.F[i][: chl * bl].view(chl, bl)
        G = chain.G[i + 2][: chr_ * br].view(chr_, br)
        b = ctx.b_effective(F, chain.B[i], chain.B[i + 1], G)
        A1 = chain.A[i][: chl * d * chm].view(chl, d, chm)
        A2 = chain.A[i + 1][: chm * d * chr_].view(chm, d, chr_)
        x0 = ctx.two_site(A1, A2)
        x = x0.clone()
        ctx.local_pcg(L, chain.W[i], chain.W[i + 1], R, b, x, abi.PRECOND_JACOBI, rtol=solve_rtol,
                      maxiter=5000)
        out.append(LocalSystem(L, chain.W[i], chain.W[i + 1], R, b, x, x0, i, N))
        ctx.sweep_range(chain, i, 1, 1, **kw)
    return out


def train(mlp: abi.Mlp, systems: list, steps: int, lr: float = 3e-3, batch: int = 0, log_every: int = 0,
          log=print) -> list:
    """Adam on the mean loss over `systems` (or over cycling mini-batches):
    one seemps_mlp_train call; returns (step, mean loss) every log_every steps."""
    losses = mlp.train(systems, steps, lr=lr, batch=batch, history=bool(log_every))
    history = []
    if log_every:
        for t, loss in enumerate(losses):
            if t % log_every == 0 or t == steps - 1:
                history.append((t, loss))
                log(f"step {t}: mean loss {loss:.4e}")
    return history


def pcg_iterations(ctx: abi.Context, systems: list, precond: int, mlp: abi.Mlp = None, rtol: float = 1e-10,
                   maxiter: int = 5000) -> tuple:
    """Total PCG iterations (and worst final residual) over the systems from their warm starts."""
    total, worst = 0, 0.0
    for s in systems:
        x = s.x0.clone()
        res, it = ctx.local_pcg(s.L, s.W1, s.W2, s.R, s.b, x, precond, rtol=rtol, maxiter=maxiter, mlp=mlp,
                                site=s.site, n_sites=s.n_sites)
        total += it
        worst = max(worst, res)
    return total, worst
