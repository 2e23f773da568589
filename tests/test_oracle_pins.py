"""Pins of the CPU oracle against what the paper and mathematics fix.

Every test here runs on the CPU (no gpu mark).  Each pin is chosen so that a
plausible slip in the oracle (a dropped term, a transposed operand, a wrong
index or sign) fails at least one of them.
"""
import os

import numpy as np
import pytest

import workloads as wl
from oracle import exact as X
from oracle import sweep as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_rows(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# ---------------------------------------------------------------- generator
def test_splitmix64_reference_vectors():
    for seed, k, val in _golden_rows("splitmix64.txt"):
        out = wl.rng.splitmix64(int(seed), int(k))[-1]
        assert int(out) == int(val, 16)


def test_gaussians_moments():
    g = wl.rng.gaussians(7, 200000)
    assert abs(g.mean()) < 0.01 and abs(g.std() - 1.0) < 0.01


# ---------------------------------------------------------------- MPO inputs
@pytest.mark.parametrize("n", [2, 3, 6])
def test_tfim_mpo_dense(n):
    H = S.mpo_to_dense(wl.mpo.tfim(n, 0.7))
    assert np.abs(H - X.tfim_dense(n, 0.7).toarray()).max() < 1e-14


def test_xxz_mpo_dense():
    H = S.mpo_to_dense(wl.mpo.xxz(7, 0.6))
    Hd = X.heisenberg_dense(7, [(i, i + 1, 1.0) for i in range(6)], 0.6).toarray()
    assert np.abs(H - Hd).max() < 1e-14


def test_graph_mpo_j1j2_dense():
    bonds = wl.mpo.j1j2_cylinder_bonds(3, 3, 1.0, 0.5)
    H = S.mpo_to_dense(wl.mpo.heisenberg_graph(9, bonds))
    assert np.abs(H - X.heisenberg_dense(9, bonds, 1.0).toarray()).max() < 1e-13
    # the graph builder on nearest-neighbour bonds reproduces the XXZ(1) chain
    Hc = S.mpo_to_dense(wl.mpo.heisenberg_graph(6, [(i, i + 1, 1.0) for i in range(5)]))
    assert np.abs(Hc - S.mpo_to_dense(wl.mpo.xxz(6, 1.0))).max() < 1e-14


@pytest.mark.parametrize("n", [1, 2, 4, 6])
def test_laplacian_1d_mpo(n):
    x, h = wl.states.interior_grid(n)
    A = S.mpo_to_dense(wl.mpo.laplacian_qtt_1d(n, h))
    N = 2 ** n
    T = (2 * np.eye(N) - np.eye(N, k=1) - np.eye(N, k=-1)) / h ** 2
    assert np.abs(A - T).max() <= 1e-14 * np.abs(T).max()
    assert max(W.shape[3] for W in wl.mpo.laplacian_qtt_1d(n, h)[:-1] or [np.zeros((1, 1, 1, 3))]) == 3


@pytest.mark.parametrize("n", [1, 2, 3])
def test_laplacian_2d_mpo(n):
    x, h = wl.states.interior_grid(n)
    Ws = wl.mpo.laplacian_qtt_2d(n, h)
    A = S.mpo_to_dense(Ws)
    N = 2 ** n
    T = (2 * np.eye(N) - np.eye(N, k=1) - np.eye(N, k=-1)) / h ** 2
    K = np.kron(T, np.eye(N)) + np.kron(np.eye(N), T)  # grid order [i_x, i_y]
    P = np.array([X.grid_to_order_b(e.reshape(N, N), n) for e in np.eye(N * N)]).T
    assert np.abs(A - P @ K @ P.T).max() <= 1e-14 * np.abs(K).max()
    assert max(W.shape[3] for W in Ws) <= 5


# ---------------------------------------------------------------- QTT inputs
def test_qtt_exact_ranks_exp_sin():
    n = 20
    x, _ = wl.states.interior_grid(n)
    for f, rank in ((np.exp(1.7 * x), 1), (np.sin(5.0 * x + 0.3), 2)):
        cores = wl.states.tt_svd(f, n, rel_tol=1e-12)
        assert max(c.shape[2] for c in cores) == rank
        assert np.abs(S.mps_to_dense(cores) - f).max() < 1e-11 * np.abs(f).max()


def test_poisson_source_mps_dense():
    n = 5
    B = wl.states.poisson_source_mps(n)
    g = X.order_b_to_grid(S.mps_to_dense(B), n)
    (f1x, f1y), (f2x, f2y) = wl.states.poisson_source_factors(n)
    F = np.outer(f1x, f1y) + np.outer(f2x, f2y)
    assert np.abs(g - F).max() < 1e-13


# ---------------------------------------------------------------- closed forms
def test_tfim_closed_form_hand_values():
    for n, g, e in _golden_rows("tfim_closed_form.txt"):
        assert abs(X.tfim_free_fermion_energy(int(n), float(g)) - float(e)) < 1e-13


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 11])
@pytest.mark.parametrize("g", [0.3, 1.0, 1.7])
def test_tfim_closed_form_vs_ed(n, g):
    e_ed = X.ground_energy(X.tfim_dense(n, g))
    assert abs(X.tfim_free_fermion_energy(n, g) - e_ed) <= 1e-12 * abs(e_ed)


def test_tfim_closed_form_vs_ed_n14():
    e_ed = X.ground_energy(X.tfim_dense(14, 1.0))
    assert abs(X.tfim_free_fermion_energy(14, 1.0) - e_ed) <= 1e-11 * abs(e_ed)


def test_tfim_bulk_energy_density():
    # E0/N -> -4/pi at g = 1 (Pfeuty 1970); the open-chain correction is O(1/N)
    n = 400
    assert abs(X.tfim_free_fermion_energy(n, 1.0) / n + 4.0 / np.pi) < 2.0 / n


def test_dirichlet_sine_eigenvectors():
    n = 6
    x, h = wl.states.interior_grid(n)
    N = 2 ** n
    T = (2 * np.eye(N) - np.eye(N, k=1) - np.eye(N, k=-1)) / h ** 2
    lam = X.dirichlet_eigenvalues(n)
    for k in (1, 3, 17):
        v = np.sin(k * np.pi * x)
        assert np.abs(T @ v - lam[k - 1] * v).max() < 1e-9 * lam[k - 1]


def test_poisson_dst_solver():
    n = 5
    x, h = wl.states.interior_grid(n)
    # sine mode: exact discrete solution
    f = np.outer(np.sin(np.pi * x), np.sin(3 * np.pi * x))
    lam = X.dirichlet_eigenvalues(n)
    u = X.poisson_dst_solve(f)
    assert np.abs(u - f / (lam[0] + lam[2])).max() < 1e-14 * np.abs(f).max() / lam[0]
    # generic source: residual of the dense 2-D stencil
    N = 2 ** n
    T = (2 * np.eye(N) - np.eye(N, k=1) - np.eye(N, k=-1)) / h ** 2
    g = np.cos(3 * x)[:, None] * np.exp(x)[None, :]
    ug = X.poisson_dst_solve(g)
    assert np.abs(T @ ug + ug @ T - g).max() < 1e-10 * np.abs(g).max()


# ---------------------------------------------------------------- local pieces
def _rand(rng, *shape):
    return rng.standard_normal(shape)


def test_heff_apply_matches_dense_and_brute_force():
    rng = np.random.default_rng(1)
    L, W1, W2, R = _rand(rng, 3, 2, 3), _rand(rng, 2, 2, 2, 3), _rand(rng, 3, 2, 2, 2), _rand(rng, 4, 2, 4)
    th = _rand(rng, 3, 2, 2, 4)
    y = S.heff_apply(L, W1, W2, R, th)
    brute = np.zeros_like(y)
    for p in range(3):
        for s1 in range(2):
            for t1 in range(2):
                for r in range(4):
                    acc = 0.0
                    for b in range(2):
                        for q in range(3):
                            for s in range(2):
                                for e in range(3):
                                    for t in range(2):
                                        for f in range(2):
                                            for c in range(4):
                                                acc += (L[p, b, q] * W1[b, s1, s, e] * W2[e, t1, t, f]
                                                        * R[r, f, c] * th[q, s, t, c])
                    brute[p, s1, t1, r] = acc
    assert np.abs(y - brute).max() < 1e-12
    Hd = S.heff_dense(L, W1, W2, R)
    assert np.abs(Hd @ th.reshape(-1) - y.reshape(-1)).max() < 1e-12
    assert np.abs(np.diag(Hd) - S.heff_diagonal(L, W1, W2, R).reshape(-1)).max() < 1e-12


def test_effective_operator_is_projected_hamiltonian():
    """H_n = P^T H P with P the isometry built from the left and right blocks."""
    n, i = 8, 3
    W = wl.mpo.xxz(n, 0.7)
    A = S.right_canonicalize(wl.states.random_mps(n, 2, 4, 3))
    # move the centre to site i by QR on sites 0..i-1
    for k in range(i):
        chl, d, chr_ = A[k].shape
        Q, Rm = np.linalg.qr(A[k].reshape(chl * d, chr_))
        A[k] = Q.reshape(chl, d, Q.shape[1])
        A[k + 1] = np.einsum("mn,nsc->msc", Rm, A[k + 1])
    Lenv = np.ones((1, 1, 1))
    for k in range(i):
        Lenv = S.left_env(Lenv, A[k], W[k])
    Renv = np.ones((1, 1, 1))
    for k in range(n - 1, i + 1, -1):
        Renv = S.right_env(Renv, A[k], W[k])
    Heff = S.heff_dense(Lenv, W[i], W[i + 1], Renv)
    Lb = A[0].reshape(-1, A[0].shape[2])
    for k in range(1, i):
        Lb = np.einsum("xa,asc->xsc", Lb, A[k]).reshape(-1, A[k].shape[2])
    Rb = A[n - 1].reshape(A[n - 1].shape[0], -1)
    for k in range(n - 2, i + 1, -1):
        Rb = np.einsum("asc,cy->asy", A[k], Rb).reshape(A[k].shape[0], -1)
    P = np.kron(np.kron(Lb, np.eye(4)), Rb.T)
    H = S.mpo_to_dense(W)
    assert np.abs(P.T @ H @ P - Heff).max() < 1e-12 * np.abs(H).max()
    assert np.abs(P.T @ P - np.eye(P.shape[1])).max() < 1e-12


def test_environments_give_expectation_and_overlap():
    rng = np.random.default_rng(5)
    n = 7
    A = wl.states.random_mps(n, 2, 5, 11)
    B = wl.states.random_mps(n, 2, 3, 12)
    W = wl.mpo.tfim(n, 0.9)
    v, w = S.mps_to_dense(A), S.mps_to_dense(B)
    H = S.mpo_to_dense(W)
    assert abs(S.expectation(A, W) - v @ H @ v) < 1e-10 * abs(v @ H @ v)
    assert abs(S.overlap(A, B) - v @ w) < 1e-10 * max(1.0, abs(v @ w))
    # right-to-left contraction gives the same number
    R = np.ones((1, 1, 1))
    G = np.ones((1, 1))
    for k in range(n - 1, -1, -1):
        R = S.right_env(R, A[k], W[k])
        G = S.right_env_linear(G, A[k], B[k])
    assert abs(R.reshape(-1)[0] - v @ H @ v) < 1e-10 * abs(v @ H @ v)
    assert abs(G.reshape(-1)[0] - v @ w) < 1e-10 * max(1.0, abs(v @ w))
    # b_n with the environments of the other sites reproduces <v, w> = a^T f
    i = 3
    F = np.ones((1, 1))
    for k in range(i):
        F = S.left_env_linear(F, A[k], B[k])
    Gr = np.ones((1, 1))
    for k in range(n - 1, i + 1, -1):
        Gr = S.right_env_linear(Gr, A[k], B[k])
    f = S.b_effective(F, B[i], B[i + 1], Gr)
    a = S.two_site(A[i], A[i + 1])
    assert abs(np.sum(a * f) - v @ w) < 1e-10 * max(1.0, abs(v @ w))


@pytest.mark.parametrize("n", [1, 2, 7, 20])
def test_lanczos_full_space_is_exact(n):
    rng = np.random.default_rng(n)
    M = rng.standard_normal((n, n))
    H = M + M.T
    e, x, m = S.lanczos_lowest(lambda v: H @ v, rng.standard_normal(n), n)
    ev = np.linalg.eigvalsh(H)
    assert abs(e - ev[0]) < 1e-12 * max(1.0, abs(ev).max())
    assert np.linalg.norm(H @ x - e * x) < 1e-10 * max(1.0, abs(ev).max())


def test_lanczos_breakdown_on_invariant_subspace():
    H = np.diag(np.arange(10.0))
    v0 = np.zeros(10)
    v0[[2, 5]] = 1.0  # Krylov space has dimension 2
    e, x, m = S.lanczos_lowest(lambda v: H @ v, v0, 8)
    assert m == 2 and abs(e - 2.0) < 1e-14


def test_truncation_rank_rules():
    s = np.array([1.0, 1e-3, 1e-7])
    assert S.truncation_rank(s, 10, 1e-12) == 2      # tail {1e-14} <= 1e-12
    assert S.truncation_rank(s, 10, 1e-15) == 3
    assert S.truncation_rank(s, 1, 1e-15) == 1       # chi_max cap
    assert S.truncation_rank(np.zeros(4), 3, 1e-12) == 1  # r >= 1
    assert S.truncation_rank(s, 10, 1e-5, S.TRUNC_RELATIVE) == 2
    rng = np.random.default_rng(3)
    for _ in range(50):
        s = np.sort(np.abs(rng.standard_normal(12)) ** 6)[::-1]
        tol = 10.0 ** rng.uniform(-8, -1)
        r = S.truncation_rank(s, 100, tol)
        tot = np.sum(s ** 2)
        assert np.sum(s[r:] ** 2) <= tol * tot * (1 + 1e-12)
        if r > 1:
            assert np.sum(s[r - 1:] ** 2) > tol * tot * (1 - 1e-12)


def test_svd_split_eckart_young():
    rng = np.random.default_rng(9)
    M = rng.standard_normal((12, 10)) @ np.diag(2.0 ** -np.arange(10))
    U, s, Vt, s_full, dw = S.svd_truncate(M, 6, 1e-30)
    assert U.shape == (12, 6)
    err2 = np.linalg.norm(M - U @ np.diag(s) @ Vt) ** 2
    assert abs(err2 / np.sum(s_full ** 2) - dw) < 1e-13
    assert np.abs(U.T @ U - np.eye(6)).max() < 1e-13
    assert np.abs(s_full - np.linalg.svd(M, compute_uv=False)).max() < 1e-13 * s_full[0]


def test_pcg_matches_direct_solve():
    rng = np.random.default_rng(2)
    M = rng.standard_normal((40, 40))
    A = M @ M.T + 40 * np.eye(40)
    b = rng.standard_normal(40)
    dg = np.diag(A)
    x, res, it = S.pcg(lambda v: A @ v, b, np.zeros(40), lambda r: r / dg, 1e-13, 200)
    xe = np.linalg.solve(A, b)
    assert np.linalg.norm(x - xe) < 1e-11 * np.linalg.norm(xe)
    assert res <= 1e-13 and 0 < it <= 40


def test_right_canonical_invariants():
    A = S.right_canonicalize(wl.states.random_mps(10, 2, 16, 4))
    for k in range(1, 10):
        assert S.right_isometry_error(A[k]) < 1e-12
    assert abs(np.linalg.norm(A[0]) - 1.0) < 1e-12
    v = S.mps_to_dense(A)
    assert abs(np.linalg.norm(v) - 1.0) < 1e-12


# ---------------------------------------------------------------- sweeps
@pytest.mark.parametrize("model", ["tfim", "xxz"])
def test_dmrg_matches_exact_diagonalisation(model):
    n = 10
    if model == "tfim":
        W = wl.mpo.tfim(n, 1.0)
        e_ex = X.tfim_free_fermion_energy(n, 1.0)
    else:
        W = wl.mpo.xxz(n, 1.0)
        e_ex = X.ground_energy(X.heisenberg_dense(n, [(i, i + 1, 1.0) for i in range(n - 1)], 1.0))
    E, A, log = S.dmrg(W, wl.states.random_mps(n, 2, 32, 0), 32, 1e-14, 4, 20)
    assert abs(E - e_ex) <= 1e-12 * abs(e_ex)
    assert abs(S.expectation(A, W) - e_ex) <= 1e-12 * abs(e_ex)
    # mixed canonical form after the last right-to-left half sweep: centre on site 0
    for k in range(1, n):
        assert S.right_isometry_error(A[k]) < 1e-12
    assert abs(np.linalg.norm(A[0]) - 1.0) < 1e-12


def test_dmrg_c1_tfim_n16():
    """The C1 workload: N=16, g=1, chi_max=32, cutoff 1e-12, 6 sweeps, k=20."""
    n = 16
    W = wl.mpo.tfim(n, 1.0)
    e_ex = X.tfim_free_fermion_energy(n, 1.0)
    E, A, log = S.dmrg(W, wl.states.random_mps(n, 2, 32, 0), 32, 1e-12, 6, 20)
    # variational: never below the exact energy; energy monotone up to truncation
    assert E >= e_ex - 1e-12 * abs(e_ex)
    assert abs(E - e_ex) <= 1e-9 * abs(e_ex)
    for a, b in zip(log.energies[1:], log.energies[:-1]):
        assert a <= b + 1e-10 * abs(e_ex)


def test_dmrg_solve_poisson_small():
    n = 4
    x, h = wl.states.interior_grid(n)
    W = wl.mpo.laplacian_qtt_2d(n, h)
    B = wl.states.poisson_source_mps(n)
    X0 = [b.copy() for b in B]
    X0[0] = 0.1 * X0[0]
    A, log = S.dmrg_solve(W, B, X0, 64, 1e-22, 4)
    u = X.order_b_to_grid(S.mps_to_dense(A), n)
    (f1x, f1y), (f2x, f2y) = wl.states.poisson_source_factors(n)
    uref = X.poisson_dst_solve(np.outer(f1x, f1y) + np.outer(f2x, f2y))
    assert np.linalg.norm(u - uref) <= 1e-10 * np.linalg.norm(uref)


def test_dmrg_solve_sine_mode_closed_form():
    n = 4
    x, h = wl.states.interior_grid(n)
    W = wl.mpo.laplacian_qtt_2d(n, h)
    B = wl.states.separable_qtt_2d([(np.sin(np.pi * x), np.sin(3 * np.pi * x))], n)
    X0 = wl.states.random_mps(2 * n, 2, 4, 5)
    A, log = S.dmrg_solve(W, B, X0, 16, 1e-22, 3)
    lam = X.dirichlet_eigenvalues(n)
    u = X.order_b_to_grid(S.mps_to_dense(A), n)
    uex = np.outer(np.sin(np.pi * x), np.sin(3 * np.pi * x)) / (lam[0] + lam[2])
    assert np.linalg.norm(u - uex) <= 1e-10 * np.linalg.norm(uex)


def test_separable_poisson_solution_matches_dst():
    # the eigen-expansion with every mode is the DST solve; with the modes of
    # a pure sine source it is the closed form at any size
    n = 8
    (f1x, f1y), (f2x, f2y) = wl.states.poisson_source_factors(n)
    u = X.poisson_dst_solve(np.outer(f1x, f1y) + np.outer(f2x, f2y))
    rng = np.random.default_rng(3)
    ix, iy = rng.integers(0, 2 ** n, 400), rng.integers(0, 2 ** n, 400)
    v = X.poisson_separable_solution(n, [(f1x, f1y), (f2x, f2y)], ix, iy, modes=2 ** n)
    assert np.abs(v - u[ix, iy]).max() <= 1e-13 * np.abs(u).max()
    n = 20
    x, h = wl.states.interior_grid(n)
    lam = X.dirichlet_eigenvalues(n)
    ix, iy = rng.integers(0, 2 ** n, 200), rng.integers(0, 2 ** n, 200)
    v = X.poisson_separable_solution(n, [(np.sin(np.pi * x), np.sin(3 * np.pi * x))], ix, iy, modes=8)
    ue = np.sin(np.pi * x[ix]) * np.sin(3 * np.pi * x[iy]) / (lam[0] + lam[2])
    assert np.abs(v - ue).max() <= 1e-13 * np.abs(ue).max()


def _sampled_sine_solve(n, extended, sweeps=2):
    x, h = wl.states.interior_grid(n)
    W = wl.mpo.laplacian_qtt_2d(n, h)
    B = wl.states.separable_qtt_2d([(np.sin(np.pi * x), np.sin(3 * np.pi * x))], n)
    X0 = [b.copy() for b in B]
    X0[0] = 0.1 * X0[0]
    A, log = S.dmrg_solve(W, B, X0, 64, 1e-24, sweeps, pcg_rtol=1e-13, pcg_maxiter=4000, extended=extended)
    u = X.order_b_to_grid(S.mps_to_dense(A), n) if n <= 6 else None
    rng = np.random.default_rng(n)
    ix, iy = rng.integers(0, 2 ** n, 2000), rng.integers(0, 2 ** n, 2000)
    vals = np.empty(len(ix))
    for k, (a, b) in enumerate(zip(ix, iy)):
        v = np.ones((1,))
        for lvl in range(n):
            v = v @ A[2 * lvl][:, (a >> (n - 1 - lvl)) & 1, :]
            v = v @ A[2 * lvl + 1][:, (b >> (n - 1 - lvl)) & 1, :]
        vals[k] = v[0]
    lam = X.dirichlet_eigenvalues(n)
    ue = np.sin(np.pi * x[ix]) * np.sin(3 * np.pi * x[iy]) / (lam[0] + lam[2])
    return np.linalg.norm(vals - ue) / np.linalg.norm(ue), u


@pytest.mark.skipif(np.finfo(np.longdouble).eps > 1e-18, reason="long double is not wider than FP64 here")
def test_dmrg_solve_extended_precision_lifts_the_fp64_floor():
    # FP64 environments of the QTT Laplacian leave ~eps 4^n / 40 (3e-10 at
    # n = 14); the extended-precision environments reach the exact discrete
    # solution far below it
    rel, _ = _sampled_sine_solve(14, extended=True)
    assert rel <= 1e-11, rel
    # and the extended mode is still the same solve: small n, dense check
    rel6, u = _sampled_sine_solve(6, extended=True)
    assert rel6 <= 1e-12, rel6
