"""Vector inputs of the sweep: random initial MPS and QTT source functions.

MPS tensors are float64 arrays A[n] of shape (chi_{n}, d, chi_{n+1}), the
storage order A[n][alpha_{n-1}, s_n, alpha_n] of Sect. 2.1, with
chi_0 = chi_N = 1.

QTT vectors follow Sect. 4.1: a function sampled on 2^n points is the tensor
v[s_1, ..., s_n] with i = 2^{n-1} s_1 + ... + s_n (most significant qubit on
the first site).  Two-dimensional functions use the interleaved order "B"
(x_1, y_1, x_2, y_2, ...).  The Dirichlet workloads sample the 2^n interior
nodes x_i = (i + 1) h of [0, 1], h = 1 / (2^n + 1), so the zero fill of the
open-boundary shift falls exactly on x = 0 and x = 1.
"""
from __future__ import annotations

import numpy as np

from .rng import gaussians, uniforms


def bond_dims(n_sites: int, d: int, chi_max: int) -> list:
    """chi_i = min(chi_max, d^i, d^(N-i)) for i = 0..N."""
    out = []
    for i in range(n_sites + 1):
        out.append(int(min(chi_max, d ** min(i, 60), d ** min(n_sites - i, 60))))
    return out


def random_mps(n_sites: int, d: int, chi_max: int, seed: int) -> list:
    """i.i.d. N(0,1) tensors drawn from one SplitMix64 stream, site 0 first,
    each tensor filled in row-major order."""
    chi = bond_dims(n_sites, d, chi_max)
    sizes = [chi[i] * d * chi[i + 1] for i in range(n_sites)]
    g = gaussians(seed, int(sum(sizes)))
    out, off = [], 0
    for i in range(n_sites):
        out.append(g[off:off + sizes[i]].reshape(chi[i], d, chi[i + 1]).copy())
        off += sizes[i]
    return out


def interior_grid(n: int) -> tuple:
    """(x, h): the 2^n interior nodes of [0, 1] and their spacing."""
    h = 1.0 / (2 ** n + 1)
    x = (np.arange(2 ** n, dtype=np.float64) + 1.0) * h
    return x, h


def tt_svd(v: np.ndarray, n: int, rel_tol: float = 1e-14) -> list:
    """Tensor-train decomposition of a length-2^n vector by sequential SVDs.

    At each cut the smallest singular values are dropped while their summed
    squares stay below (rel_tol * ||v||)^2 / (n - 1).  This builds inputs
    only; it is not the sweep's split.
    """
    v = np.asarray(v, dtype=np.float64)
    norm2 = float(v @ v)
    budget = (rel_tol ** 2) * norm2 / max(1, n - 1)
    cores = []
    r = 1
    M = v.reshape(r * 2, -1)
    for k in range(n - 1):
        U, s, Vt = np.linalg.svd(M, full_matrices=False)
        tail = np.cumsum((s ** 2)[::-1])[::-1]  # tail[j] = sum_{i>=j} s_i^2
        keep = len(s)
        for j in range(1, len(s)):
            if tail[j] <= budget:
                keep = j
                break
        cores.append(U[:, :keep].reshape(r, 2, keep))
        M = (s[:keep, None] * Vt[:keep]).reshape(keep * 2, -1)
        r = keep
    cores.append(M.reshape(r, 2, 1))
    return cores


def interleave(X: list, Y: list) -> list:
    """MPS of f(x) g(y) in order B from 1-D MPS X (of f) and Y (of g)."""
    n = len(X)
    assert len(Y) == n
    out = []
    for k in range(n):
        ax0, ax1 = X[k].shape[0], X[k].shape[2]
        by0, by1 = Y[k].shape[0], Y[k].shape[2]
        # x site: bond (alpha_{k-1}, beta_{k-1}) -> (alpha_k, beta_{k-1})
        Cx = np.einsum("asc,bd->abscd", X[k], np.eye(by0))
        Cx = Cx.reshape(ax0 * by0, 2, ax1 * by0)
        # y site: bond (alpha_k, beta_{k-1}) -> (alpha_k, beta_k)
        Cy = np.einsum("ac,bse->absce", np.eye(ax1), Y[k])
        Cy = Cy.reshape(ax1 * by0, 2, ax1 * by1)
        out.extend([Cx, Cy])
    return out


def mps_direct_sum(A: list, B: list) -> list:
    """MPS of a + b: concatenated end tensors, block-diagonal bulk tensors."""
    n = len(A)
    out = []
    for k in range(n):
        a, b = A[k], B[k]
        if n == 1:
            out.append(a + b)
        elif k == 0:
            out.append(np.concatenate([a, b], axis=2))
        elif k == n - 1:
            out.append(np.concatenate([a, b], axis=0))
        else:
            C = np.zeros((a.shape[0] + b.shape[0], a.shape[1], a.shape[2] + b.shape[2]))
            C[: a.shape[0], :, : a.shape[2]] = a
            C[a.shape[0]:, :, a.shape[2]:] = b
            out.append(C)
    return out


def poisson_source_factors(n: int, centre=(0.3, 0.6), sigma=0.05, kx=1, ky=3):
    """Separable factors of f = sin(kx pi x) sin(ky pi y) + exp(-|r - r0|^2 / (2 sigma^2)).

    Returns ((f1x, f1y), (f2x, f2y)) sampled on the interior grid; the
    Gaussian has unit peak.
    """
    x, _ = interior_grid(n)
    f1x = np.sin(kx * np.pi * x)
    f1y = np.sin(ky * np.pi * x)
    f2x = np.exp(-((x - centre[0]) ** 2) / (2 * sigma ** 2))
    f2y = np.exp(-((x - centre[1]) ** 2) / (2 * sigma ** 2))
    return (f1x, f1y), (f2x, f2y)


def separable_qtt_2d(terms: list, n: int, rel_tol: float = 1e-14) -> list:
    """Order-B MPS of sum_t fx_t(x) fy_t(y) from sampled 1-D factors."""
    parts = []
    for fx, fy in terms:
        parts.append(interleave(tt_svd(fx, n, rel_tol), tt_svd(fy, n, rel_tol)))
    out = parts[0]
    for p in parts[1:]:
        out = mps_direct_sum(out, p)
    return out


def poisson_source_mps(n: int, rel_tol: float = 1e-14) -> list:
    """The C4 right-hand side f on the 2^n x 2^n interior grid as an order-B MPS."""
    t1, t2 = poisson_source_factors(n)
    return separable_qtt_2d([t1, t2], n, rel_tol)


def random_poisson_source_terms(n: int, seed: int) -> list:
    """Random source: 1-4 Gaussians plus one low sine mode, as separable factors.

    Centres in U(0.15, 0.85)^2, widths in U(0.03, 0.2), amplitudes N(0,1),
    sine mode (kx, ky) uniform in {1..4}^2 with an N(0,1) amplitude.
    """
    u = uniforms(seed, 32)
    g = gaussians(seed ^ 0x5DEECE66D, 8)
    x, _ = interior_grid(n)
    count = 1 + int(u[0] * 4) % 4
    terms = []
    for t in range(count):
        cx = 0.15 + 0.7 * u[1 + 3 * t]
        cy = 0.15 + 0.7 * u[2 + 3 * t]
        sg = 0.03 + 0.17 * u[3 + 3 * t]
        amp = g[t]
        terms.append((amp * np.exp(-((x - cx) ** 2) / (2 * sg ** 2)),
                      np.exp(-((x - cy) ** 2) / (2 * sg ** 2))))
    kx = 1 + int(u[20] * 4) % 4
    ky = 1 + int(u[21] * 4) % 4
    terms.append((g[5] * np.sin(kx * np.pi * x), np.sin(ky * np.pi * x)))
    return terms
