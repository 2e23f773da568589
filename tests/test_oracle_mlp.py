"""Pins of the learned-preconditioner oracle (oracle/mlp.py)."""
import numpy as np

import workloads as wl
from oracle import mlp as M
from oracle import sweep as S


def _system(seed=0, chl=3, chr_=4, D=3, d=2):
    rng = np.random.default_rng(seed)
    L = rng.standard_normal((chl, D, chl))
    L = np.einsum("aBc,dBc->aBd", L, L) + 0.5  # positive blocks
    R = rng.standard_normal((chr_, D, chr_))
    R = np.einsum("aBc,dBc->aBd", R, R) + 0.5
    W1 = np.abs(rng.standard_normal((D, d, d, D)))
    W1 = 0.5 * (W1 + W1.transpose(0, 2, 1, 3))
    W2 = np.abs(rng.standard_normal((D, d, d, D)))
    W2 = 0.5 * (W2 + W2.transpose(0, 2, 1, 3))
    A = S.heff_dense(L, W1, W2, R)
    A = 0.5 * (A + A.T)
    A = A + np.eye(A.shape[0]) * (abs(np.linalg.eigvalsh(A)[0]) + 1.0)  # SPD
    shape = (chl, d, d, chr_)
    diag = np.diag(A).reshape(shape).copy()
    b = rng.standard_normal(shape)
    xstar = np.linalg.solve(A, b.reshape(-1)).reshape(shape)
    Aop = lambda v: (A @ v.reshape(-1)).reshape(v.shape)
    return L, R, A, diag, b, xstar, Aop


def test_init_is_jacobi():
    L, R, A, diag, b, xstar, Aop = _system()
    theta = M.init_params(3)
    X = M.features(diag, L, R, 2, 10)
    o, _ = M.forward(theta, X)
    p, U = M.precond_factors(o, diag)
    assert np.allclose(p * diag.reshape(-1), 1.0, rtol=1e-14)
    assert np.abs(U).max() == 0.0


def test_precond_is_spd():
    L, R, A, diag, b, xstar, Aop = _system(1)
    rng = np.random.default_rng(4)
    theta = rng.standard_normal(M.param_count()) * 0.3
    o, _ = M.forward(theta, M.features(diag, L, R, 1, 6))
    p, U = M.precond_factors(o, diag)
    P = np.diag(p) + U @ U.T
    assert np.linalg.eigvalsh(P)[0] > 0
    r = rng.standard_normal(p.size)
    assert np.allclose(M.apply_precond(p, U, r), P @ r, rtol=1e-13, atol=1e-14)


def test_loss_definition_dense():
    L, R, A, diag, b, xstar, Aop = _system(2)
    rng = np.random.default_rng(5)
    theta = rng.standard_normal(M.param_count()) * 0.2
    X = M.features(diag, L, R, 3, 8)
    loss, _ = M.loss_and_grad(theta, X, diag, b, xstar, Aop)
    o, _ = M.forward(theta, X)
    p, U = M.precond_factors(o, diag)
    P = np.diag(p) + U @ U.T
    e = xstar.reshape(-1) - P @ b.reshape(-1)
    xs = xstar.reshape(-1)
    assert abs(loss - (e @ A @ e) / (xs @ A @ xs)) < 1e-12 * max(1.0, loss)


def test_gradient_matches_central_differences():
    L, R, A, diag, b, xstar, Aop = _system(3)
    rng = np.random.default_rng(6)
    theta = rng.standard_normal(M.param_count()) * 0.2
    X = M.features(diag, L, R, 3, 8)
    _, g = M.loss_and_grad(theta, X, diag, b, xstar, Aop)
    h = 1e-6
    idx = rng.choice(theta.size, 60, replace=False)
    idx = np.concatenate([idx, [0, theta.size - 1, theta.size - 5, 7 * 64 + 3]])
    for k in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        fd = (M.loss_and_grad(tp, X, diag, b, xstar, Aop)[0] -
              M.loss_and_grad(tm, X, diag, b, xstar, Aop)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(g[k])) + 1e-9, (k, fd, g[k])


def test_adam_first_step_is_signed_lr():
    theta = np.array([1.0, -2.0, 0.5])
    grad = np.array([0.3, -4.0, 1e-3])
    m, v = np.zeros(3), np.zeros(3)
    out = M.adam_step(theta.copy(), grad, m, v, 1, 0.01, eps=0.0)
    assert np.allclose(out, np.array([1.0, -2.0, 0.5]) - 0.01 * np.sign(grad), rtol=1e-14)


def test_adam_three_steps_hand_sequence():
    """Three Adam steps (beta1 0.9, beta2 0.999, lr 0.1, eps 0) worked by hand
    in decimal arithmetic.  Entry 0: g = 0.5, -0.25, 0.1 from theta = 1:
      t=1: m = 0.05, v = 0.00025, m^ = 0.05/0.1 = 0.5, v^ = 0.00025/0.001 = 0.25,
           theta = 1 - 0.1 * 0.5/0.5 = 0.9
      t=2: m = 0.045 - 0.025 = 0.02, v = 0.00024975 + 0.0000625 = 0.00031225,
           m^ = 0.02/0.19, v^ = 0.00031225/0.001999,
           theta = 0.9 - 0.1 * 0.105263157894737 / sqrt(0.156203101550775) = 0.873366296033960
      t=3: m = 0.018 + 0.01 = 0.028, v = 0.00031193775 + 0.00001 = 0.00032193775,
           m^ = 0.028/0.271, v^ = 0.00032193775/0.002997001,
           theta = 0.841841939389988
    Entry 1: g = 2, 2, -1 from theta = -2: a constant gradient moves by lr
    each step (-2.1, -2.2), then m = 0.342 - 0.1 = 0.242, v = 0.007988004 +
    0.001 = 0.008988004, theta = -2.251565340578533.  A wrong moment update
    or bias correction after the first step changes steps 2 and 3."""
    theta = np.array([1.0, -2.0])
    m, v = np.zeros(2), np.zeros(2)
    grads = [np.array([0.5, 2.0]), np.array([-0.25, 2.0]), np.array([0.1, -1.0])]
    expect = [np.array([0.9, -2.1]), np.array([0.8733662960339597, -2.2]),
              np.array([0.8418419393899876, -2.2515653405785326])]
    for t, (g, e) in enumerate(zip(grads, expect), 1):
        theta = M.adam_step(theta, g, m, v, t, 0.1, eps=0.0)
        assert np.allclose(theta, e, rtol=1e-14, atol=0), (t, theta, e)
    assert np.allclose(m, [0.028, 0.242], rtol=1e-14) and np.allclose(v, [0.00032193775, 0.008988004], rtol=1e-13)


def test_features_values():
    L, R, A, diag, b, xstar, Aop = _system(4, chl=2, chr_=3)
    X = M.features(diag, L, R, 5, 10).reshape(2, 2, 2, 3, M.N_FEAT)
    assert np.allclose(X[..., 0], np.log10(diag) / 10)
    assert np.allclose(X[..., 1], 0.5) and np.allclose(X[..., 2], 0.6)
    assert np.allclose(X[1, :, :, :, 3], np.log10(np.linalg.norm(L[1, :, 1])) / 10)
    assert np.allclose(X[:, :, :, 2, 4], np.log10(np.linalg.norm(R[2, :, 2])) / 10)
    assert np.all(X[:, 1, :, :, 5] == 1.0) and np.all(X[:, :, 0, :, 6] == 0.0)
