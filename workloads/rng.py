"""Counter-based SplitMix64 generator and the Gaussian draws built on it.

SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014): the k-th output (k = 1, 2, ...) of the stream with
seed s is mix(s + k * 0x9E3779B97F4A7C15), where mix is the published
xor-shift/multiply finaliser.  Because every output is a pure function of
(seed, k) the generator is counter-based and vectorises in numpy.

Doubles in [0, 1) take the top 53 bits of an output.  Gaussians use the
Box-Muller transform on consecutive pairs (u1, u2): the pair yields
sqrt(-2 ln(1-u1)) * (cos(2 pi u2), sin(2 pi u2)).

This module holds no arithmetic of the sweep itself; both the oracle and the
CUDA path read the arrays it produces.
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Outputs number offset+1 ... offset+count of the SplitMix64 stream."""
    k = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniforms(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits of each output."""
    z = splitmix64(seed, count, offset)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def gaussians(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """count standard normal draws (Box-Muller over consecutive uniform pairs).

    The draws are consumed in pairs: gaussian 2j and 2j+1 come from uniforms
    2j and 2j+1 of the stream (after `offset` pairs have been skipped).
    """
    npairs = (count + 1) // 2
    u = uniforms(seed, 2 * npairs, 2 * offset)
    u1 = 1.0 - u[0::2]  # in (0, 1]
    u2 = u[1::2]
    rad = np.sqrt(-2.0 * np.log(u1))
    out = np.empty(2 * npairs)
    out[0::2] = rad * np.cos(2.0 * np.pi * u2)
    out[1::2] = rad * np.sin(2.0 * np.pi * u2)
    return out[:count]
