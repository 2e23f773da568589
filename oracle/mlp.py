"""Learned local preconditioner for the PCG solve of the sweep: plain FP64 NumPy.

TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and the CPU-baseline
leg of the benchmark may import this module; the CUDA path never does.

The paper leaves the solver of the local system U_n a_n = b_n of
DMRG-as-solver open (Sect. 3.2.3: a standard iterative method); it has no
learned part.  The preconditioner here is an addition, defined as follows:

* per-entry features of the local system at the pair (i, i+1) of an N-site
  chain, for the entry (a, s, t, c):
    x0 = log10(diag_j) / 10, x1 = i / N, x2 = (i + 1) / N,
    x3 = log10(|L[a, :, a]|) / 10, x4 = log10(|R[c, :, c]|) / 10,
    x5 = s / (d - 1), x6 = t / (d - 1)
  (diag = the diagonal of the effective operator, |.| the 2-norm over the
  MPO index; d = 1 gives x5 = x6 = 0);
* a multilayer perceptron x -> tanh(W1 x + b1) -> tanh(W2 h1 + b2) ->
  o = W3 h2 + b3 with five outputs;
* p_j = softplus(o0_j) / diag_j and U_jk = o_{1+k, j} / sqrt(n) (k < 4);
  the preconditioner P = diag(p) + U U^T is symmetric positive definite;
* loss of one system with exact solution x*: |x* - P b|_A^2 / (x*^T b),
  the A-norm error of one preconditioned step from zero, relative to
  |x*|_A^2 = x*^T A x* = x*^T b.

Parameters are one flat float vector in the order W1 (64 x 7), b1, W2
(64 x 64), b2, W3 (5 x 64), b3 (row-major weights, out x in).
"""
from __future__ import annotations

import numpy as np

N_FEAT = 7
N_OUT = 5
RANK = 4


def param_count(hidden: int = 64) -> int:
    return hidden * N_FEAT + hidden + hidden * hidden + hidden + N_OUT * hidden + N_OUT


def unpack(theta: np.ndarray, hidden: int = 64):
    o = 0
    out = []
    for shape in ((hidden, N_FEAT), (hidden,), (hidden, hidden), (hidden,), (N_OUT, hidden), (N_OUT,)):
        n = int(np.prod(shape))
        out.append(theta[o:o + n].reshape(shape))
        o += n
    return out


def softplus(x):
    return np.where(x > 20, x, np.log1p(np.exp(np.minimum(x, 20))))


def sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def features(diag, L, R, site: int, n_sites: int) -> np.ndarray:
    """Per-entry features, shape (n_loc, 7), entries in (a, s, t, c) order."""
    chl, d, _, chr_ = diag.shape
    Ln = np.linalg.norm(np.einsum("aba->ab", L), axis=1)  # |L[a, :, a]|
    Rn = np.linalg.norm(np.einsum("cfc->cf", R), axis=1)
    X = np.zeros((chl, d, d, chr_, N_FEAT))
    X[..., 0] = np.log10(diag) / 10.0
    X[..., 1] = site / n_sites
    X[..., 2] = (site + 1) / n_sites
    X[..., 3] = (np.log10(Ln + 1e-300) / 10.0)[:, None, None, None]
    X[..., 4] = (np.log10(Rn + 1e-300) / 10.0)[None, None, None, :]
    if d > 1:
        X[..., 5] = (np.arange(d) / (d - 1))[None, :, None, None]
        X[..., 6] = (np.arange(d) / (d - 1))[None, None, :, None]
    return X.reshape(-1, N_FEAT)


def forward(theta, X, hidden: int = 64):
    """Returns (o, cache) with o of shape (n, 5)."""
    W1, b1, W2, b2, W3, b3 = unpack(theta, hidden)
    a1 = X @ W1.T + b1
    h1 = np.tanh(a1)
    a2 = h1 @ W2.T + b2
    h2 = np.tanh(a2)
    o = h2 @ W3.T + b3
    return o, (X, h1, h2)


def precond_factors(o, diag):
    """p (n,) and U (n, 4) from the network outputs."""
    n = o.shape[0]
    p = softplus(o[:, 0]) / diag.reshape(-1)
    U = o[:, 1:1 + RANK] / np.sqrt(n)
    return p, U


def apply_precond(p, U, r):
    """z = P r = p * r + U (U^T r)."""
    return p * r + U @ (U.T @ r)


def loss_and_grad(theta, X, diag, b, xstar, Aop, hidden: int = 64):
    """Loss of one system and its gradient with respect to theta.

    Aop(v) applies the local operator A.  With q = P b, e = x* - q,
    loss = e^T A e / (x*^T b); dloss/dq = -2 A e / (x*^T b) = g;
    dloss/dp_j = g_j b_j; dloss/dU_jk = g_j (U^T b)_k + b_j (U^T g)_k;
    then the chain rule through softplus, the 1/sqrt(n) scale and the two
    tanh layers.
    """
    W1, b1, W2, b2, W3, b3 = unpack(theta, hidden)
    bb = b.reshape(-1)
    xs = xstar.reshape(-1)
    dg = diag.reshape(-1)
    n = bb.size
    o, (Xc, h1, h2) = forward(theta, X, hidden)
    p, U = precond_factors(o, diag)
    w = U.T @ bb
    q = p * bb + U @ w
    e = xs - q
    Ae = Aop(e.reshape(b.shape)).reshape(-1)
    D = float(xs @ bb)
    loss = float(e @ Ae) / D
    g = -2.0 * Ae / D
    dp = g * bb
    Utg = U.T @ g
    dU = np.outer(g, w) + np.outer(bb, Utg)
    do = np.zeros_like(o)
    do[:, 0] = dp * sigmoid(o[:, 0]) / dg
    do[:, 1:1 + RANK] = dU / np.sqrt(n)
    # backprop through the layers
    dW3 = do.T @ h2
    db3 = do.sum(axis=0)
    dh2 = do @ W3
    da2 = dh2 * (1.0 - h2 * h2)
    dW2 = da2.T @ h1
    db2 = da2.sum(axis=0)
    dh1 = da2 @ W2
    da1 = dh1 * (1.0 - h1 * h1)
    dW1 = da1.T @ Xc
    db1 = da1.sum(axis=0)
    grad = np.concatenate([dW1.ravel(), db1, dW2.ravel(), db2, dW3.ravel(), db3])
    return loss, grad


def init_params(seed: int, hidden: int = 64) -> np.ndarray:
    """Seeded initialisation that starts exactly at the Jacobi preconditioner:
    small random hidden weights, W3 = 0, b3 = (softplus^{-1}(1), 0, 0, 0, 0),
    so p = 1/diag and U = 0 before training."""
    from workloads.rng import gaussians

    g = gaussians(seed, param_count(hidden))
    theta = np.zeros(param_count(hidden))
    W1, b1, W2, b2, W3, b3 = unpack(theta, hidden)
    o = 0
    W1[:] = g[o:o + W1.size].reshape(W1.shape) * np.sqrt(1.0 / N_FEAT)
    o += W1.size
    W2[:] = g[o:o + W2.size].reshape(W2.shape) * np.sqrt(1.0 / hidden)
    o += W2.size
    b3[0] = np.log(np.expm1(1.0))
    return theta


def adam_step(theta, grad, m, v, t: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015), bias-corrected; t counts from 1."""
    m[:] = beta1 * m + (1 - beta1) * grad
    v[:] = beta2 * v + (1 - beta2) * grad * grad
    mh = m / (1 - beta1 ** t)
    vh = v / (1 - beta2 ** t)
    theta[:] = theta - lr * mh / (np.sqrt(vh) + eps)
    return theta
