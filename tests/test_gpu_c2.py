"""The Heisenberg XXZ chain of the chi = 1024 benchmark at the bond dimension
the CPU oracle can reach (chi_max = 256): Delta = 1, N = 100, MPO bond 5,
random MPS from seed 1, weight cutoff 1e-12, Krylov dimension 20, full
sweeps of the whole chain.  The reference is the oracle's own run of the
same configuration for 10 sweeps, stored by tests/golden/make_c2_chi256.py
(its energy is converged to 1e-14 relative after the fourth half sweep).

Bounds: the FP64 GPU path within 1e-10 of the oracle's energy, the mixed
path (bf16x3 contractions, 10 sweeps) followed by one FP64 refinement sweep
within 1e-9; both variational with respect to it up to those bounds."""
import os

import numpy as np
import pytest

import workloads as wl
from oracle import sweep as S

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "c2_xxz_n100_chi256.txt")
N, CHI = 100, 256


def golden():
    out = {}
    with open(GOLDEN) as fh:
        for line in fh:
            parts = line.split()
            if parts and not line.startswith("#") and parts[0] != "half":
                out[parts[0]] = float(parts[1])
    return out


@pytest.fixture(scope="module")
def pkg():
    import torch
    assert torch.cuda.is_available()
    import paper_2601_16734_gb300 as pkg
    pkg.build()
    return pkg


@pytest.fixture(scope="module")
def ctx(pkg):
    c = pkg.Context(0, chi_max=CHI, d=2, D_max=5, krylov_dim=20)
    yield c
    assert c.device_status() == 0
    c.close()


def run(pkg, ctx, precision, sweeps, refine):
    W = wl.mpo.xxz(N, 1.0)
    ch = pkg.Chain(ctx, W, wl.states.random_mps(N, 2, CHI, 1), CHI)
    rep = ctx.sweep(ch, mode=pkg.MODE_EIG, n_sweeps=sweeps, refine_sweeps=refine, precision=precision,
                    krylov_dim=20, chi_max=CHI, tol=1e-12)
    A = [t.cpu().numpy() for t in ch.tensors()]
    return rep, A, W


def test_c2_chi256_fp64_vs_oracle(ctx, pkg):
    ref = golden()
    rep, A, W = run(pkg, ctx, pkg.FP64, 4, 0)
    e, e_or = rep["energy"], ref["final_energy"]
    print(f"C2 chi=256 FP64 GPU (4 sweeps): {e!r} vs oracle {e_or!r}: rel {abs(e - e_or) / abs(e_or):.2e}")
    assert abs(e - e_or) <= 1e-10 * abs(e_or)
    # the reported energy is the state's energy: <psi|H|psi> by the oracle's own contraction
    assert abs(S.expectation(A, W) - e) <= 1e-10 * abs(e_or)


def test_c2_chi256_mixed_then_fp64_refinement_vs_oracle(ctx, pkg):
    ref = golden()
    rep, A, W = run(pkg, ctx, pkg.BF16X3, 10, 1)
    e, e_or = rep["energy"], ref["final_energy"]
    e_mixed = rep["half_sweep_energy"][19]  # last half sweep before the refinement
    print(f"C2 chi=256 bf16x3 x10 + FP64 x1: {e!r} vs oracle {e_or!r}: rel {abs(e - e_or) / abs(e_or):.2e} "
          f"(before refinement {abs(e_mixed - e_or) / abs(e_or):.2e})")
    assert abs(e - e_or) <= 1e-9 * abs(e_or)
    assert abs(S.expectation(A, W) - e) <= 1e-9 * abs(e_or)
