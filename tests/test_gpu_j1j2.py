"""J1-J2 cylinder (the C5 model) at a size the oracle and exact diagonalisation
finish quickly: width 4 x length 3 (12 sites), J2/J1 = 0.5, exact
finite-state-machine MPO (bond dimension up to 2 + 3 x open sites, so the MPO
mixing runs through the wide-block path of the contraction kernels).

chi_max = 64 = 2^(N/2) makes the two-site sweep exact, so the FP64 GPU sweep
must reach the exact ground energy, agree with the oracle's sweep, and the
mixed-precision sweep plus one FP64 refinement sweep must agree with both.
"""
import numpy as np
import pytest

import workloads as wl
from oracle import exact as X
from oracle import sweep as S

pytestmark = pytest.mark.gpu

WIDTH, LENGTH = 4, 3
N = WIDTH * LENGTH
CHI = 64


@pytest.fixture(scope="module")
def pkg():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_2601_16734_gb300 as pkg
    pkg.build()
    return pkg


@pytest.fixture(scope="module")
def model():
    bonds = wl.mpo.j1j2_cylinder_bonds(WIDTH, LENGTH, 1.0, 0.5)
    W = wl.mpo.heisenberg_graph(N, bonds)
    return bonds, W


@pytest.fixture(scope="module")
def ctx(pkg, model):
    _, W = model
    D_max = max(max(w.shape[0], w.shape[3]) for w in W)
    c = pkg.Context(0, chi_max=CHI, d=2, D_max=D_max, krylov_dim=20)
    yield c
    assert c.device_status() == 0
    c.close()


def _sweep(ctx, pkg, W, A0, n_sweeps, precision, refine=0):
    ch = pkg.Chain(ctx, W, A0, CHI)
    rep = ctx.sweep(ch, mode=pkg.MODE_EIG, n_sweeps=n_sweeps, refine_sweeps=refine, precision=precision,
                    krylov_dim=20, chi_max=CHI, tol=1e-14)
    return rep, [t.detach().cpu().numpy() for t in ch.tensors()]


def test_mpo_is_wide(model):
    _, W = model
    assert max(w.shape[3] for w in W) * 4 > 32  # D d^2 above the register mixing limit


def test_j1j2_fp64_sweep_exact(ctx, pkg, model):
    bonds, W = model
    A0 = wl.states.random_mps(N, 2, CHI, 2)
    rep, A = _sweep(ctx, pkg, W, A0, 4, pkg.FP64)
    e_ed = X.ground_energy(X.heisenberg_dense(N, bonds))
    assert abs(rep["energy"] - e_ed) <= 1e-9 * abs(e_ed)
    assert abs(S.expectation(A, W) - e_ed) <= 1e-9 * abs(e_ed)
    e_or, _, _ = S.dmrg(W, A0, CHI, 1e-14, 4, 20)
    assert abs(rep["energy"] - e_or) <= 1e-10 * abs(e_or)


def test_j1j2_mixed_with_refinement(ctx, pkg, model):
    bonds, W = model
    A0 = wl.states.random_mps(N, 2, CHI, 2)
    rep, _ = _sweep(ctx, pkg, W, A0, 3, pkg.BF16X3, refine=1)
    e_ed = X.ground_energy(X.heisenberg_dense(N, bonds))
    assert abs(rep["energy"] - e_ed) <= 1e-9 * abs(e_ed)
