"""Pins of the oracle's variational compression (Sect. 2.3; Sect. 2.4.1, eq. of psi_opt;
sums of MPS as in Sect. 2.4.1) against what the mathematics fixes:

- with enough bond dimension the compression reproduces b exactly;
- on two sites it is the truncated SVD of the dense tensor (Eckart-Young);
- a weighted sum of MPS, passed as its direct sum, is reproduced exactly;
- the distance from overlaps equals the distance of the dense vectors;
- after a pair update x is a truncated orthogonal projection of b.
"""
import numpy as np

import workloads as wl
from oracle import sweep as S


def _dense(A):
    return S.mps_to_dense(A).reshape(-1)


def test_distance2_matches_dense():
    a = wl.states.random_mps(8, 2, 6, 11)
    b = wl.states.random_mps(8, 2, 5, 12)
    assert abs(S.distance2(a, b) - np.sum((_dense(a) - _dense(b)) ** 2)) <= 1e-12 * np.sum(_dense(b) ** 2)


def test_simplify_exact_when_bond_suffices():
    b = wl.states.random_mps(10, 2, 8, 3)
    x0 = wl.states.random_mps(10, 2, 8, 4)
    x, log = S.simplify(b, x0, 8, 1e-30, 2)
    rel = np.linalg.norm(_dense(x) - _dense(b)) / np.linalg.norm(_dense(b))
    assert rel < 1e-12
    assert S.distance2(x, b) <= 1e-22 * S.overlap(b, b)


def test_simplify_two_sites_is_truncated_svd():
    rng = np.random.default_rng(7)
    B = [rng.standard_normal((1, 4, 3)), rng.standard_normal((3, 4, 1))]
    x0 = [rng.standard_normal((1, 4, 2)), rng.standard_normal((2, 4, 1))]
    x, _ = S.simplify(B, x0, 2, 1e-30, 1)
    M = (B[0].reshape(4, 3) @ B[1].reshape(3, 4))
    s = np.linalg.svd(M, compute_uv=False)
    assert abs(S.distance2(x, B) - np.sum(s[2:] ** 2)) <= 1e-12 * np.sum(s ** 2)
    U, sv, Vt = np.linalg.svd(M)
    best = (U[:, :2] * sv[:2]) @ Vt[:2]
    assert np.linalg.norm(_dense(x).reshape(4, 4) - best) <= 1e-12 * np.linalg.norm(M)


def test_simplify_weighted_sum_of_mps():
    p1 = wl.states.random_mps(9, 2, 4, 21)
    p2 = wl.states.random_mps(9, 2, 3, 22)
    w1, w2 = 0.7, -1.3
    q1 = [t.copy() for t in p1]
    q1[0] = w1 * q1[0]
    q2 = [t.copy() for t in p2]
    q2[0] = w2 * q2[0]
    b = wl.states.mps_direct_sum(q1, q2)
    x, _ = S.simplify(b, wl.states.random_mps(9, 2, 7, 23), 7, 1e-30, 2)
    target = w1 * _dense(p1) + w2 * _dense(p2)
    assert np.linalg.norm(_dense(x) - target) <= 1e-11 * np.linalg.norm(target)


def test_simplify_truncated_is_a_projection():
    """Compressing below b's bond dimension: after a pair update x is the
    truncated orthogonal projection of b onto the pair's space, so
    <b, x> = |x|^2 and |b - x|^2 = |b|^2 - |x|^2 > 0."""
    b = wl.states.random_mps(10, 2, 16, 5)
    x, log = S.simplify(b, wl.states.random_mps(10, 2, 6, 6), 6, 1e-30, 3)
    nb, nx, bx = S.overlap(b, b), S.overlap(x, x), S.overlap(b, x)
    assert abs(bx - nx) <= 1e-12 * nb
    d2 = S.distance2(x, b)
    assert d2 > 1e-6 * nb
    assert abs(d2 - (nb - nx)) <= 1e-12 * nb
