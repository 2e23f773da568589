"""Seeded synthetic inputs shared by the oracle and the CUDA path.

Holds the counter-based generator, the operator (MPO) builders and the vector
(MPS / QTT) builders.  None of the sweep's own arithmetic lives here.
"""
from . import rng, mpo, states  # noqa: F401
