"""CPU oracle of the two-site variational sweep (plain FP64 NumPy).

TEST INFRASTRUCTURE ONLY.  This package exists to check the CUDA path.  Only
tests/, __graft_entry__.smoke() and the cpu_baseline / reference legs of
bench.py may import or run anything in it; the library under
paper_2601_16734_gb300/ never imports it and shares no code with it.

Modules:
  sweep  - environments, effective operator, Lanczos, PCG, truncated SVD,
           canonical form, the DMRG and DMRG-solve sweeps (Sects. 2.3, 2.4,
           3.1.1, 3.2.3).
  exact  - exact diagonalisation, the free-fermion closed form of the open
           transverse-field Ising chain, the DST Poisson solver.
  mlp    - forward/backward of the learned local preconditioner.

Parity status: every function here is pinned by a `-m "not gpu"` test in
tests/test_oracle_*.py against a value fixed by the paper or by mathematics
(closed forms, brute force, invariants, textbook library routines).
"""
from . import sweep, exact, mlp  # noqa: F401
