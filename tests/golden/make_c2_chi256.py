"""Writes c2_xxz_n100_chi256.txt: the CPU oracle's two-site DMRG on the
Heisenberg XXZ chain (Delta = 1, N = 100, Pauli products, MPO bond 5) from the
seeded random MPS (seed 1) at chi_max = 256, weight cutoff 1e-12, Krylov
dimension 20, 10 sweeps: the energy after every half sweep, the largest
discarded weight of every half sweep, the accumulated truncation bound, and
<psi|H|psi> of the final MPS by full contraction.

Calls only oracle/ and workloads/ (about an hour of CPU).  Run from the
repository root:  python tests/golden/make_c2_chi256.py
"""
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import workloads as wl  # noqa: E402
from oracle import sweep as S  # noqa: E402

N, CHI, SEED, SWEEPS, K, TOL = 100, 256, 1, 10, 20, 1e-12


def main():
    t0 = time.time()
    W = wl.mpo.xxz(N, 1.0)
    A0 = wl.states.random_mps(N, 2, CHI, SEED)
    E, A, log = S.dmrg(W, A0, CHI, TOL, SWEEPS, K)
    Eexp = S.expectation(A, W)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "c2_xxz_n100_chi256.txt")
    with open(out, "w") as fh:
        fh.write("# CPU oracle (oracle.sweep.dmrg), XXZ Delta=1 N=100 d=2 D=5, random MPS seed 1,\n")
        fh.write(f"# chi_max={CHI}, weight cutoff {TOL}, Krylov {K}, {SWEEPS} sweeps; written by make_c2_chi256.py\n")
        fh.write("# half_sweep energy max_discarded_weight\n")
        for h, (e, dw) in enumerate(zip(log.energies, log.discarded)):
            fh.write(f"half {h} {e!r} {dw!r}\n")
        fh.write(f"final_energy {E!r}\n")
        fh.write(f"expectation {Eexp!r}\n")
        fh.write(f"error_bound {log.error!r}\n")
        fh.write(f"max_rank {max(max(r) for r in log.ranks)}\n")
    print(f"wrote {out} in {time.time() - t0:.0f} s: E = {E!r}")


if __name__ == "__main__":
    main()
