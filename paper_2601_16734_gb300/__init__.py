"""GB300 (sm_103a) implementation of the two-site variational sweep of the
SeeMPS MPS/TT method: DMRG eigen-search, DMRG linear solve, variational
compression, two-site TDVP and the variational MPO-MPS product.

The compute path is libseemps_gb300.so (hand-written CUDA, C ABI declared in
include/seemps_gb300.h); `abi` is its thin ctypes binding.  There is no CPU
fallback: loading fails loudly if the library cannot be built or loaded.
"""
from .abi import (  # noqa: F401
    ABSORB_LEFT, ABSORB_RIGHT, BF16X3, FP64, FP64X2, LEFT, MODE_EIG, MODE_APPLY, MODE_SIMPLIFY, MODE_SOLVE, MODE_TDVP,
    PRECOND_JACOBI, PRECOND_MLP, PRECOND_NONE, RIGHT, TRUNC_RELATIVE, TRUNC_WEIGHT, Chain, Context, SeempsError,
    Mlp, load, workspace_bytes,
)
from ._build import build, lib_path  # noqa: F401
