"""Pins of the oracle's MPO-MPS product (Sect. 2.4.2, matrix-vector product:
the enlarged tensors of eq. C and the variational problem
argmin |w - U v|^2) against what the mathematics fixes:

- the enlarged-tensor MPS equals the dense H b;
- the mixed environments give <x, U b> of the dense vectors;
- with enough bond dimension the variational product is U b exactly;
- on two sites it is the truncated SVD of U b (Eckart-Young);
- it equals the variational compression of the explicit product (the same
  local vectors through a different contraction);
- after a pair update x is a truncated projection: <U b, x> = |x|^2.
"""
import numpy as np

import workloads as wl
from oracle import sweep as S


def _dense(A):
    return S.mps_to_dense(A).reshape(-1)


def test_product_mps_is_dense_product():
    W = wl.mpo.xxz(7, 0.6)
    b = wl.states.random_mps(7, 2, 5, 1)
    v = _dense(S.mpo_mps_product(W, b))
    ref = S.mpo_to_dense(W) @ _dense(b)
    assert np.linalg.norm(v - ref) <= 1e-12 * np.linalg.norm(ref)


def test_mixed_environments_give_the_form():
    n = 6
    W = wl.mpo.tfim(n, 0.7)
    x = wl.states.random_mps(n, 2, 3, 2)
    b = wl.states.random_mps(n, 2, 4, 3)
    ref = _dense(x) @ (S.mpo_to_dense(W) @ _dense(b))
    L = np.ones((1, 1, 1))
    for i in range(n):
        L = S.left_env_mixed(L, x[i], W[i], b[i])
    R = np.ones((1, 1, 1))
    for i in range(n - 1, -1, -1):
        R = S.right_env_mixed(R, x[i], W[i], b[i])
    assert abs(L.item() - ref) <= 1e-12 * abs(ref)
    assert abs(R.item() - ref) <= 1e-12 * abs(ref)


def test_apply_exact_when_bond_suffices():
    n = 8
    W = wl.mpo.xxz(n, 1.0)
    b = wl.states.random_mps(n, 2, 4, 5)
    x, _ = S.apply_mpo(W, b, wl.states.random_mps(n, 2, 20, 6), 20, 1e-30, 2)
    ref = S.mpo_to_dense(W) @ _dense(b)
    assert np.linalg.norm(_dense(x) - ref) <= 1e-11 * np.linalg.norm(ref)


def test_apply_two_sites_is_truncated_svd():
    rng = np.random.default_rng(8)
    W = [rng.standard_normal((1, 3, 3, 2)), rng.standard_normal((2, 3, 3, 1))]
    b = [rng.standard_normal((1, 3, 3)), rng.standard_normal((3, 3, 1))]
    x, _ = S.apply_mpo(W, b, [rng.standard_normal((1, 3, 2)), rng.standard_normal((2, 3, 1))], 2, 1e-30, 1)
    M = (S.mpo_to_dense(W) @ _dense(b)).reshape(3, 3)
    U, sv, Vt = np.linalg.svd(M)
    best = (U[:, :2] * sv[:2]) @ Vt[:2]
    assert np.linalg.norm(_dense(x).reshape(3, 3) - best) <= 1e-12 * np.linalg.norm(M)


def test_apply_equals_compression_of_the_product():
    n = 10
    W = wl.mpo.xxz(n, 0.8)
    b = wl.states.random_mps(n, 2, 6, 9)
    x0 = wl.states.random_mps(n, 2, 7, 10)
    x, _ = S.apply_mpo(W, b, x0, 7, 1e-30, 2)
    y, _ = S.simplify(S.mpo_mps_product(W, b), x0, 7, 1e-30, 2)
    assert np.linalg.norm(_dense(x) - _dense(y)) <= 1e-10 * np.linalg.norm(_dense(y))


def test_apply_truncated_is_a_projection():
    n = 10
    W = wl.mpo.tfim(n, 1.2)
    b = wl.states.random_mps(n, 2, 8, 11)
    x, _ = S.apply_mpo(W, b, wl.states.random_mps(n, 2, 5, 12), 5, 1e-30, 2)
    ub = S.mpo_to_dense(W) @ _dense(b)
    v = _dense(x)
    nu, nx, ux = ub @ ub, v @ v, ub @ v
    assert abs(ux - nx) <= 1e-12 * nu
    d2 = np.sum((ub - v) ** 2)
    assert d2 > 1e-8 * nu
    assert abs(d2 - (nu - nx)) <= 1e-12 * nu
