"""Pins of the oracle's global conjugate gradients on MPS (Sect. 3.2.1, the
CGS listing of Fig. cgs) and of the joined sum it builds on (Sect. 2.4.1):

- the joined MPS of a weighted sum is the weighted sum of the dense vectors;
- with a bond dimension that holds every vector exactly (2^(N/2)), the MPS
  iterates are textbook conjugate gradients on the dense system step by step
  (a wrong alpha, an unsquared beta or a wrong sign shows at step 2);
- run to convergence it solves U x = b (numpy.linalg.solve).
The operator is U = shift I + tridiag(-1, 2, -1), symmetric positive definite
with condition number (4 + shift) / shift at most.
"""
import numpy as np

import workloads as wl
from oracle import sweep as S


def _dense(A):
    return S.mps_to_dense(A).reshape(-1)


def _shifted_laplacian(n, shift):
    """tridiag(-1, 2, -1) + shift I as an MPO: the QTT Laplacian with h = 1 and
    the shift added to its no-carry (identity) channel on the last site."""
    W = wl.mpo.laplacian_qtt_1d(n, 1.0)
    W[-1] = W[-1].copy()
    W[-1][0, :, :, 0] += shift * np.eye(2)
    return W


def _dense_cg(U, b, x0, steps):
    x = x0.copy()
    r = b - U @ x
    p = r.copy()
    for _ in range(steps):
        a = (r @ r) / (p @ U @ p)
        x = x + a * p
        r_new = b - U @ x
        p = r_new + (r_new @ r_new) / (r @ r) * p
        r = r_new
    return x


def test_mps_sum_is_the_weighted_sum():
    A = wl.states.random_mps(7, 2, 4, 1)
    B = wl.states.random_mps(7, 2, 3, 2)
    C = wl.states.random_mps(7, 2, 5, 3)
    w = [0.7, -1.3, 2.1]
    v = _dense(S.mps_sum(w, [A, B, C]))
    ref = w[0] * _dense(A) + w[1] * _dense(B) + w[2] * _dense(C)
    assert np.linalg.norm(v - ref) <= 1e-12 * np.linalg.norm(ref)


def test_operator_is_the_shifted_stencil():
    n = 5
    U = S.mpo_to_dense(_shifted_laplacian(n, 0.5))
    m = 2 ** n
    ref = np.diag(np.full(m, 2.5)) - np.diag(np.ones(m - 1), 1) - np.diag(np.ones(m - 1), -1)
    assert np.abs(U - ref).max() <= 1e-14


def test_iterates_are_textbook_cg():
    n = 6
    W = _shifted_laplacian(n, 0.5)
    U = S.mpo_to_dense(W)
    b = wl.states.random_mps(n, 2, 4, 4)
    x0 = wl.states.random_mps(n, 2, 3, 5)
    for steps in (1, 2, 3):
        x, _, k, _ = S.cgs_solve(W, b, x0, 8, 1e-30, 0.0, steps)
        assert k == steps
        ref = _dense_cg(U, _dense(b), _dense(x0), steps)
        assert np.linalg.norm(_dense(x) - ref) <= 1e-10 * np.linalg.norm(ref)


def test_converges_to_the_solution():
    n = 6
    W = _shifted_laplacian(n, 0.5)
    U = S.mpo_to_dense(W)
    b = wl.states.random_mps(n, 2, 4, 6)
    x, res, k, hist = S.cgs_solve(W, b, wl.states.random_mps(n, 2, 2, 7), 8, 1e-30, 1e-10, 100)
    nb = np.linalg.norm(_dense(b))
    assert res < 1e-10 * nb and k < 100
    ref = np.linalg.solve(U, _dense(b))
    assert np.linalg.norm(_dense(x) - ref) <= 1e-9 * np.linalg.norm(ref)
    assert hist[-1] == res and hist[0] > res


def test_zero_right_hand_side_stops_at_zero():
    """b = 0 from x0 = 0: |r| = 0 at once, no step is taken and x stays 0."""
    n = 5
    W = _shifted_laplacian(n, 0.5)
    b = [0.0 * t for t in wl.states.random_mps(n, 2, 2, 15)]
    x0 = [0.0 * t for t in wl.states.random_mps(n, 2, 2, 16)]
    x, res, k, _ = S.cgs_solve(W, b, x0, 4, 1e-30, 1e-10, 10)
    assert res == 0.0 and k == 0
    assert np.abs(_dense(x)).max() == 0.0
