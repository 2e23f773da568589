"""Pins of the oracle's two-site TDVP (Sect. 7.3, TDVP; generator L = -H) and its
pieces against what the mathematics fixes:

- the one-site effective operator reproduces <psi|H|psi> for a state whose
  centre sits on that site (a non-trivial left environment);
- the Krylov exponential with the full Krylov space equals scipy's expm;
- on two sites the step is the exact normalised exp(-dt H) psi, and at the
  full bond dimension every step is (the manifold is the whole space);
- long imaginary-time evolution reaches the exact ground energy.
"""
import numpy as np
import scipy.linalg

import workloads as wl
from oracle import exact as X
from oracle import sweep as S


def _dense(A):
    v = S.mps_to_dense(A).reshape(-1)
    return v / np.linalg.norm(v)


def test_one_site_operator_gives_the_energy():
    n = 6
    W = wl.mpo.xxz(n, 0.7)
    A = S.right_canonicalize(wl.states.random_mps(n, 2, 4, 8))
    # move the centre to site 1 with a QR of site 0
    a0 = A[0].reshape(-1, A[0].shape[2])
    Q, Rm = np.linalg.qr(a0)
    A[0] = Q.reshape(A[0].shape[0], A[0].shape[1], Q.shape[1])
    A[1] = np.einsum("ij,jsk->isk", Rm, A[1])
    L1 = S.left_env(np.ones((1, 1, 1)), A[0], W[0])
    R2 = np.ones((1, 1, 1))
    for i in range(n - 1, 1, -1):
        R2 = S.right_env(R2, A[i], W[i])
    e_local = float(np.vdot(A[1], S.heff1_apply(L1, W[1], R2, A[1])))
    e_full = S.expectation(A, W)
    assert abs(e_local - e_full) <= 1e-12 * abs(e_full)


def test_krylov_expm_full_space_is_exact():
    rng = np.random.default_rng(3)
    H = rng.standard_normal((12, 12))
    H = 0.5 * (H + H.T)
    v = rng.standard_normal(12)
    for tau in (-0.3, 0.2):
        x, m, a0 = S.krylov_expm(lambda u: H @ u, v, tau, 30)
        ref = scipy.linalg.expm(tau * H) @ v
        assert m == 12
        assert np.linalg.norm(x - ref) <= 1e-11 * np.linalg.norm(ref)
        assert abs(a0 - v @ H @ v / (v @ v)) <= 1e-12 * abs(a0)


def test_two_sites_is_exact_evolution():
    W = wl.mpo.tfim(2, 0.8)
    A0 = wl.states.random_mps(2, 2, 2, 4)
    H = S.mpo_to_dense(W)
    dt = 0.37
    _, A, _ = S.tdvp(W, A0, dt, 1, 4, 1e-30, 10)
    ref = scipy.linalg.expm(-dt * H) @ _dense(A0)
    ref /= np.linalg.norm(ref)
    v = _dense(A)
    assert np.linalg.norm(v - np.sign(v @ ref) * ref) <= 1e-12


def test_exact_at_full_bond_dimension():
    """With the bond dimension of the whole Hilbert space the MPS manifold is
    the whole space and the projected evolution is the exact one: several
    steps of any dt reproduce exp(-t H) psi (a wrong sign or order of the
    backward one-site step would leave an O(dt) error)."""
    n = 6
    W = wl.mpo.tfim(n, 1.1)
    A0 = wl.states.random_mps(n, 2, 8, 5)
    H = S.mpo_to_dense(W)
    for dt, steps in ((0.1, 4), (0.35, 2)):
        ref = scipy.linalg.expm(-dt * steps * H) @ _dense(A0)
        ref /= np.linalg.norm(ref)
        _, A, _ = S.tdvp(W, A0, dt, steps, 8, 1e-30, 20)
        v = _dense(A)
        assert np.linalg.norm(v - np.sign(v @ ref) * ref) <= 1e-11


def test_imaginary_time_reaches_the_ground_state():
    n = 8
    W = wl.mpo.tfim(n, 1.0)
    E, _, _ = S.tdvp(W, wl.states.random_mps(n, 2, 16, 6), 0.5, 60, 16, 1e-14, 20)
    e_ed = X.ground_energy(X.tfim_dense(n, 1.0))
    assert abs(E - e_ed) <= 1e-9 * abs(e_ed)


# ---- real time (generator L = -i H, complex tensors)

def test_krylov_expm_real_time_full_space_is_exact():
    """With the whole space as Krylov space the Lanczos exponential with an
    imaginary tau is exp(-i t H) v, for a real and for a complex start vector."""
    rng = np.random.default_rng(21)
    n = 12
    H = rng.standard_normal((n, n))
    H = H + H.T
    for v in (rng.standard_normal(n), rng.standard_normal(n) + 1j * rng.standard_normal(n)):
        t = 0.73
        x, m, _ = S.krylov_expm(lambda y: H @ y, v, -1j * t, n, 1e-15)
        ref = scipy.linalg.expm(-1j * t * H) @ v
        assert m == n
        assert np.linalg.norm(x - ref) <= 1e-12 * np.linalg.norm(ref)


def _dense_c(A):
    v = S.mps_to_dense(A).reshape(-1)
    return v / np.linalg.norm(v)


def test_real_time_two_sites_is_exact_evolution():
    """One real-time step on two sites is exp(-i dt H) psi itself: the pair is
    the whole state and no one-site step follows the last pair."""
    W = wl.mpo.tfim(2, 0.8)
    A0 = wl.states.random_mps(2, 2, 2, 4)
    H = S.mpo_to_dense(W)
    dt = 0.37
    _, A, _ = S.tdvp(W, A0, dt, 1, 4, 1e-30, 10, real_time=True)
    ref = scipy.linalg.expm(-1j * dt * H) @ _dense_c(A0)
    assert np.linalg.norm(_dense_c(A) - ref) <= 1e-12


def test_real_time_exact_at_full_bond_dimension():
    """At the bond dimension of the whole Hilbert space the projected
    real-time evolution is the exact one: several steps of any dt reproduce
    exp(-i t H) psi, phase included (a wrong sign of either the forward or
    the backward step would leave an O(dt) error); the norm and the energy
    are conserved."""
    n = 6
    W = wl.mpo.xxz(n, 0.6)
    A0 = wl.states.random_mps(n, 2, 8, 5)
    H = S.mpo_to_dense(W)
    psi0 = _dense_c(A0)
    e0 = float(np.real(np.vdot(psi0, H @ psi0)))
    for dt, steps in ((0.1, 4), (0.35, 2)):
        ref = scipy.linalg.expm(-1j * dt * steps * H) @ psi0
        E, A, _ = S.tdvp(W, A0, dt, steps, 8, 1e-30, 20, real_time=True)
        v = S.mps_to_dense(A).reshape(-1)
        assert abs(np.linalg.norm(v) - 1.0) <= 1e-12
        assert np.linalg.norm(v - ref) <= 1e-11
        assert abs(E - e0) <= 1e-11 * abs(e0)
