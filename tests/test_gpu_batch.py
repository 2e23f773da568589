"""Batched DMRG over independent transverse-field Ising chains of uneven
length and bond dimension (the C3 workload shape, scaled to test size):
every chain's energy against its free-fermion closed form, and every
batched result equal to the same chain swept alone."""
import time

import numpy as np
import pytest

import workloads as wl
from oracle import exact as X

pytestmark = pytest.mark.gpu


def chain_specs(count, seed=3):
    """g ~ U[0.5, 1.5], N ~ U{16..40}, chi_max ~ U{16, 32, 64} from SplitMix64(seed + index)."""
    out = []
    for k in range(count):
        u = wl.rng.uniforms(seed + k, 3)
        out.append((0.5 + u[0], 16 + int(u[1] * 25), [16, 32, 64][int(u[2] * 3)]))
    return out


def test_batched_tfim_chains_match_closed_form_and_solo_runs():
    import torch
    import paper_2601_16734_gb300 as pkg
    from paper_2601_16734_gb300 import abi
    pkg.build()
    specs = chain_specs(12)
    ctxs, chains, params = [], [], []
    for k, (g, n, chi) in enumerate(specs):
        ctxs.append(pkg.Context(0, chi_max=chi, d=2, D_max=3, krylov_dim=20,
                                stream=torch.cuda.Stream()))
        chains.append(pkg.Chain(ctxs[-1], wl.mpo.tfim(n, g), wl.states.random_mps(n, 2, chi, 100 + k), chi))
        params.append(dict(mode=pkg.MODE_EIG, n_sweeps=4, refine_sweeps=1, precision=pkg.BF16X3,
                           krylov_dim=20, chi_max=chi, tol=1e-12))
    torch.cuda.synchronize()  # chain buffers were filled on torch's stream
    t0 = time.time()
    reps = abi.sweep_batch(ctxs, chains, params, max_threads=12)
    t_batch = time.time() - t0
    worst = 0.0
    for (g, n, chi), rep in zip(specs, reps):
        e_ff = X.tfim_free_fermion_energy(n, g)
        rel = abs(rep["energy"] - e_ff) / abs(e_ff)
        worst = max(worst, rel)
        assert rep["energy"] >= e_ff - 1e-10 * abs(e_ff)  # variational
        # 1e-9 relative to the closed form, plus what the chain's own truncation
        # at chi_max (its logged largest discarded weight) can account for
        assert rel <= 1e-9 + 10 * rep["max_discarded"], (g, n, chi, rel, rep["max_discarded"])
    # the same chains alone, one after the other
    t0 = time.time()
    for k, (g, n, chi) in enumerate(specs):
        ch = pkg.Chain(ctxs[k], wl.mpo.tfim(n, g), wl.states.random_mps(n, 2, chi, 100 + k), chi)
        torch.cuda.synchronize()
        rep = ctxs[k].sweep(ch, **params[k])
        assert rep["energy"] == reps[k]["energy"]
    t_solo = time.time() - t0
    print(f"{len(specs)} chains: batched {t_batch:.2f} s, one by one {t_solo:.2f} s, "
          f"worst relative energy error {worst:.2e}")
    for c in ctxs:
        assert c.device_status() == 0
        c.close()


def test_batch_rejects_shared_context():
    import torch
    import paper_2601_16734_gb300 as pkg
    from paper_2601_16734_gb300 import abi
    ctx = pkg.Context(0, chi_max=8, d=2, D_max=3)
    ch = [pkg.Chain(ctx, wl.mpo.tfim(6, 1.0), wl.states.random_mps(6, 2, 8, k), 8) for k in range(2)]
    torch.cuda.synchronize()
    with pytest.raises(abi.SeempsError):
        abi.sweep_batch([ctx, ctx], ch, [dict(chi_max=8), dict(chi_max=8)])
    ctx.close()
