"""Exact references the sweep is checked against.

TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and the CPU-baseline
leg of the benchmark may import this module; the CUDA path never does.

* Exact diagonalisation by brute force: the Hamiltonian assembled from
  Kronecker products of Pauli matrices, site 0 the most significant factor.
* Open transverse-field Ising chain H = -sum Z Z - g sum X (Pauli): after the
  Jordan-Wigner map the ground energy is minus the sum of the singular values
  of the N x N upper-bidiagonal matrix with g on the diagonal and 1 above it.
* Dirichlet Poisson on the interior grid x_i = (i+1) h, h = 1/(2^n + 1): the
  vectors sin(k pi x_i) are eigenvectors of the 3-point stencil (2 v_i -
  v_{i+1} - v_{i-1})/h^2 with eigenvalue (4/h^2) sin^2(k pi h / 2), so a
  type-I discrete sine transform diagonalises the 2-D operator exactly.
"""
from __future__ import annotations

import numpy as np
import scipy.fft
import scipy.sparse as sp
import scipy.sparse.linalg as spla

_X = sp.csr_matrix(np.array([[0.0, 1.0], [1.0, 0.0]]))
_Y_IM = sp.csr_matrix(np.array([[0.0, -1.0], [1.0, 0.0]]))  # Y = i * _Y_IM
_Z = sp.csr_matrix(np.array([[1.0, 0.0], [0.0, -1.0]]))


def _site_op(op, i: int, n: int):
    left = sp.identity(2 ** i, format="csr")
    right = sp.identity(2 ** (n - i - 1), format="csr")
    return sp.kron(sp.kron(left, op, format="csr"), right, format="csr")


def tfim_dense(n: int, g: float):
    """Sparse H = -sum_i Z_i Z_{i+1} - g sum_i X_i."""
    H = sp.csr_matrix((2 ** n, 2 ** n))
    for i in range(n - 1):
        H = H - _site_op(_Z, i, n) @ _site_op(_Z, i + 1, n)
    for i in range(n):
        H = H - g * _site_op(_X, i, n)
    return H


def heisenberg_dense(n: int, bonds: list, delta: float = 1.0):
    """Sparse H = sum J (X X + Y Y + delta Z Z) over the given (i, j, J) bonds.

    Y_i Y_j = (i Y')(i Y') = -Y' Y' with Y' the real antisymmetric part.
    """
    H = sp.csr_matrix((2 ** n, 2 ** n))
    for (i, j, c) in bonds:
        H = H + c * (_site_op(_X, i, n) @ _site_op(_X, j, n)
                     - _site_op(_Y_IM, i, n) @ _site_op(_Y_IM, j, n)
                     + delta * _site_op(_Z, i, n) @ _site_op(_Z, j, n))
    return H


def ground_energy(H) -> float:
    """Lowest eigenvalue: dense eigh up to dimension 4096, else ARPACK."""
    if H.shape[0] <= 4096:
        return float(np.linalg.eigvalsh(H.toarray())[0])
    vals = spla.eigsh(H, k=1, which="SA", tol=1e-14, maxiter=100000)[0]
    return float(vals[0])


def tfim_free_fermion_energy(n: int, g: float) -> float:
    """Closed-form ground energy of the open Pauli TFIM chain."""
    T = np.diag(np.full(n, float(g))) + np.diag(np.ones(n - 1), 1)
    return -float(np.sum(np.linalg.svd(T, compute_uv=False)))


def dirichlet_eigenvalues(n: int) -> np.ndarray:
    """lambda_k = (4/h^2) sin^2(k pi h/2), k = 1..2^n, for the interior grid."""
    h = 1.0 / (2 ** n + 1)
    k = np.arange(1, 2 ** n + 1, dtype=np.float64)
    return (4.0 / h ** 2) * np.sin(k * np.pi * h / 2.0) ** 2


def poisson_dst_solve(f2d: np.ndarray) -> np.ndarray:
    """Exact discrete solution of (A_x + A_y) u = f by the type-I DST.

    f2d[i_x, i_y] sampled on the interior grid.  DST-I with orthonormal
    scaling is its own inverse.
    """
    nx = int(round(np.log2(f2d.shape[0])))
    ny = int(round(np.log2(f2d.shape[1])))
    lx = dirichlet_eigenvalues(nx)
    ly = dirichlet_eigenvalues(ny)
    fh = scipy.fft.dstn(f2d, type=1, norm="ortho")
    uh = fh / (lx[:, None] + ly[None, :])
    return scipy.fft.idstn(uh, type=1, norm="ortho")


def poisson_separable_solution(n: int, terms: list, ix, iy, modes: int = 1024) -> np.ndarray:
    """Exact discrete solution of (A_x + A_y) u = sum_t fx_t (x) fy_t at grid points.

    The Dirichlet stencil's eigenvectors are s_j(i) = sqrt(2/(N+1)) sin(j pi (i+1) h),
    j = 1..N = 2^n, with eigenvalues lambda_j (dirichlet_eigenvalues), so
    u(i_x, i_y) = sum_t sum_{j,k} fx^_j fy^_k s_j(i_x) s_k(i_y) / (lambda_j + lambda_k)
    with fx^ = DST-I(fx) (orthonormal, the same transform as poisson_dst_solve).
    The double sum runs over j, k <= `modes`; for smooth factors the
    coefficients decay fast and the tail is below rounding (the caller checks
    it by doubling `modes`).  ix, iy: integer grid indices of the points.
    """
    N = 2 ** n
    J = min(modes, N)
    lam = dirichlet_eigenvalues(n)[:J]
    h = 1.0 / (N + 1)
    j = np.arange(1, J + 1, dtype=np.float64)
    ix = np.asarray(ix, dtype=np.float64)
    iy = np.asarray(iy, dtype=np.float64)
    Sx = np.sqrt(2.0 / (N + 1)) * np.sin(np.pi * h * np.outer(ix + 1.0, j))  # [P, J]
    Sy = np.sqrt(2.0 / (N + 1)) * np.sin(np.pi * h * np.outer(iy + 1.0, j))
    out = np.zeros(len(ix))
    denom = lam[:, None] + lam[None, :]
    for fx, fy in terms:
        cx = scipy.fft.dst(np.asarray(fx, dtype=np.float64), type=1, norm="ortho")[:J]
        cy = scipy.fft.dst(np.asarray(fy, dtype=np.float64), type=1, norm="ortho")[:J]
        Cm = np.outer(cx, cy) / denom
        out += np.einsum("pj,jk,pk->p", Sx, Cm, Sy, optimize=True)
    return out


def order_b_to_grid(v: np.ndarray, n: int) -> np.ndarray:
    """Dense order-B vector (x_1, y_1, ..., x_n, y_n bits) -> array [i_x, i_y]."""
    T = v.reshape([2] * (2 * n))
    perm = list(range(0, 2 * n, 2)) + list(range(1, 2 * n, 2))
    return np.transpose(T, perm).reshape(2 ** n, 2 ** n)


def grid_to_order_b(u: np.ndarray, n: int) -> np.ndarray:
    """Array [i_x, i_y] -> dense order-B vector."""
    T = u.reshape([2] * (2 * n))
    perm = []
    for k in range(n):
        perm += [k, n + k]
    return np.transpose(T, perm).reshape(-1)
