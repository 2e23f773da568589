"""Plain FP64 restatement of the two-site variational sweep.

TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and the CPU-baseline
leg of the benchmark may import this module; the CUDA path never does.

Every function follows the paper's definitions in its own notation:

* MPS tensors A[n][alpha_{n-1}, s_n, alpha_n] (Sect. 2.1) and MPO tensors
  B[n][beta_{n-1}, j_n, i_n, beta_n] with j the output index (Sect. 2.2).
* Environments of the quadratic form <v, H w> (Sect. 2.5): the left one is
  L[a', b, a] (bra bond, MPO bond, ket bond) and contracts sites 0..n-1; the
  right one is R[c', f, c] and contracts sites n+2..N-1.  The antilinear form
  <v, w> has environments F[a, a''] (v bond, w bond) and G[c, c''].
* The local problem on the pair (n, n+1) acts on the two-site vector
  a_n[a, s, t, c] = sum_m A_n[a, s, m] A_{n+1}[m, t, c] (Sect. 2.5).
* Canonical form and truncation (Sect. 2.3), DMRG (Sect. 3.1.1) and DMRG as
  a linear solver (Sect. 3.2.3), each sweep visiting the pairs from the left
  end to the right end and back (Sect. 2.5); variational compression
  (Sect. 2.3), the variational MPO-MPS product (Sect. 2.4.2) and two-site TDVP
  (Sect. 7.3) on the same sweep; global conjugate gradients on MPS built from
  them (Sect. 3.2.1).

Where the paper is silent the reading taken is stated next to the code that
takes it.  einsum is used as a library contraction primitive; every call
spells out the paper's index sum.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

TRUNC_WEIGHT = "weight"      # discarded squared weight <= tol * total weight
TRUNC_RELATIVE = "relative"  # keep s_j > tol * s_0 (Sect. 2.3)


# --------------------------------------------------------------------------
# dense helpers (small sizes only)
# --------------------------------------------------------------------------
def mps_to_dense(A: list) -> np.ndarray:
    """v_{s_1...s_L} = A^(1)s_1 ... A^(L)s_L, the MPS of Eq. (general-MPS)."""
    v = A[0]
    for T in A[1:]:
        v = np.tensordot(v, T, axes=([v.ndim - 1], [0]))
    return v.reshape(-1)


def mpo_to_dense(W: list) -> np.ndarray:
    """U^{j_1..j_L}_{i_1..i_L} = B^(1) ... B^(L), the MPO of Eq. (MPO)."""
    T = W[0]  # (1, j, i, D)
    n = 1
    for B in W[1:]:
        T = np.tensordot(T, B, axes=([T.ndim - 1], [0]))
        n += 1
    # axes: 1, j1, i1, j2, i2, ..., jL, iL, 1
    T = T.reshape(T.shape[1:-1])
    perm = list(range(0, 2 * n, 2)) + list(range(1, 2 * n, 2))
    T = np.transpose(T, perm)
    d = int(round(T.size ** (1.0 / (2 * n))))
    dim = int(np.prod(T.shape[:n]))
    return T.reshape(dim, dim)


# --------------------------------------------------------------------------
# environments (Sect. 2.5, quadratic and antilinear forms)
# --------------------------------------------------------------------------
def left_env(L: np.ndarray, A: np.ndarray, W: np.ndarray) -> np.ndarray:
    """L_{n+1}[c', f, c] = sum conj(A[a', s', c']) L_n[a', b, a] W[b, s', s, f] A[a, s, c].

    Evaluated as three pairwise index sums: over a, then over (b, s), then
    over (a', s').
    """
    T = np.einsum("pbq,qsc->pbsc", L, A, optimize=True)  # T[a', b, s, c]
    T = np.einsum("pbsc,bjsf->pjcf", T, W, optimize=True)  # T[a', s', c, f]
    return np.einsum("pjcf,pjr->rfc", T, A.conj(), optimize=True)


def right_env(R: np.ndarray, A: np.ndarray, W: np.ndarray) -> np.ndarray:
    """R_n[a', b, a] = sum conj(A[a', s', c']) W[b, s', s, f] R_{n+1}[c', f, c] A[a, s, c].

    Evaluated as three pairwise index sums: over c, then over (s, f), then
    over (s', c').
    """
    T = np.einsum("rfc,qsc->rfqs", R, A, optimize=True)  # T[c', f, a, s]
    T = np.einsum("rfqs,bjsf->rqbj", T, W, optimize=True)  # T[c', a, b, s']
    return np.einsum("rqbj,pjr->pbq", T, A.conj(), optimize=True)


def left_env_linear(F: np.ndarray, A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """F_{n+1}[c, c''] = sum conj(A[a, s, c]) F_n[a, a''] B[a'', s, c'']."""
    T = np.einsum("ab,bsd->asd", F, B, optimize=True)
    return np.einsum("asd,asc->cd", T, A.conj(), optimize=True)


def right_env_linear(G: np.ndarray, A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """G_n[a, a''] = sum conj(A[a, s, c]) G_{n+1}[c, c''] B[a'', s, c'']."""
    T = np.einsum("cd,bsd->cbs", G, B, optimize=True)
    return np.einsum("cbs,asc->ab", T, A.conj(), optimize=True)


# --------------------------------------------------------------------------
# local operators on the two-site vector
# --------------------------------------------------------------------------
def two_site(A1: np.ndarray, A2: np.ndarray) -> np.ndarray:
    """a_n[a, s, t, c] = sum_m A_n[a, s, m] A_{n+1}[m, t, c]."""
    return np.einsum("asm,mtc->astc", A1, A2, optimize=True)


def heff_apply(L, W1, W2, R, theta) -> np.ndarray:
    """(H_n a)[a', s', t', c'] = sum L[a', b, a] W1[b, s', s, e] W2[e, t', t, f] R[c', f, c] a[a, s, t, c].

    Evaluated as four pairwise index sums: over a, over (b, s), over (e, t),
    over (c, f).
    """
    T = np.einsum("pbq,qstc->pbstc", L, theta, optimize=True)  # T[a', b, s, t, c]
    T = np.einsum("pbstc,bjse->pjtce", T, W1, optimize=True)  # T[a', s', t, c, e]
    T = np.einsum("pjtce,ektf->pjkcf", T, W2, optimize=True)  # T[a', s', t', c, f]
    return np.einsum("pjkcf,rfc->pjkr", T, R, optimize=True)  # y[a', s', t', c']


def heff_dense(L, W1, W2, R) -> np.ndarray:
    """H_n as an explicit (n_loc x n_loc) matrix, rows = output index."""
    H = np.einsum("pbq,bsue,etvf,rfw->pstrquvw", L, W1, W2, R)
    n = L.shape[0] * W1.shape[1] * W2.shape[1] * R.shape[0]
    return H.reshape(n, n)


def heff_diagonal(L, W1, W2, R) -> np.ndarray:
    """diag(H_n)[a, s, t, c] = sum_{b,e,f} L[a, b, a] W1[b, s, s, e] W2[e, t, t, f] R[c, f, c]."""
    Ld = np.einsum("aba->ab", L)
    W1d = np.einsum("bsse->bse", W1)
    W2d = np.einsum("ettf->etf", W2)
    Rd = np.einsum("cfc->cf", R)
    T = np.einsum("ab,bse->ase", Ld, W1d, optimize=True)
    T = np.einsum("ase,etf->astf", T, W2d, optimize=True)
    return np.einsum("astf,cf->astc", T, Rd, optimize=True)


def b_effective(F, B1, B2, G) -> np.ndarray:
    """f_n[a, s, t, c] = sum F[a, a''] B_n[a'', s, e] B_{n+1}[e, t, c''] G[c, c'']."""
    T = np.einsum("ax,xse->ase", F, B1, optimize=True)
    T = np.einsum("ase,etz->astz", T, B2, optimize=True)
    return np.einsum("astz,cz->astc", T, G, optimize=True)


# --------------------------------------------------------------------------
# truncation (Sect. 2.3)
# --------------------------------------------------------------------------
def truncation_rank(s: np.ndarray, chi_max: int, tol: float, mode: str = TRUNC_WEIGHT) -> int:
    """Number of singular values kept, r >= 1.

    weight mode: the smallest r with sum_{j>=r} s_j^2 <= tol * sum_j s_j^2,
    both sums accumulated one term at a time from the smallest value upward
    (fixed order, so equal inputs give equal ranks bit for bit), capped at
    chi_max.  relative mode: the number of s_j > tol * s_0, capped at chi_max.
    s must be sorted in descending order.
    """
    n = len(s)
    if n == 0:
        return 0
    if mode == TRUNC_RELATIVE:
        thr = tol * float(s[0])
        r = 0
        for j in range(n):
            if float(s[j]) > thr:
                r += 1
        return max(1, min(chi_max, r))
    sq = [float(x) * float(x) for x in s]
    total = 0.0
    for j in range(n - 1, -1, -1):
        total = total + sq[j]
    limit = tol * total
    # tail(r) = sum_{j >= r} s_j^2; scan r downward while tail(r) <= limit
    r = n
    tail = 0.0
    for j in range(n - 1, 0, -1):
        tail = tail + sq[j]
        if tail <= limit:
            r = j
        else:
            break
    return max(1, min(chi_max, r))


def svd_truncate(M: np.ndarray, chi_max: int, tol: float, mode: str = TRUNC_WEIGHT):
    """Truncated SVD M ~= U_r S_r V_r^T; returns U_r, s_r, Vt_r, s (full), discarded weight.

    The discarded weight is sum_{j>=r} s_j^2 / sum_j s_j^2.
    """
    try:
        U, s, Vt = np.linalg.svd(M, full_matrices=False)
    except np.linalg.LinAlgError:  # gesdd failure: fall back to gesvd
        import scipy.linalg
        U, s, Vt = scipy.linalg.svd(M, full_matrices=False, lapack_driver="gesvd")
    r = truncation_rank(s, chi_max, tol, mode)
    total = float(np.sum(s * s))
    dw = float(np.sum(s[r:] ** 2)) / total if total > 0 else 0.0
    return U[:, :r], s[:r], Vt[:r], s, dw


# --------------------------------------------------------------------------
# canonical form (Sect. 2.3)
# --------------------------------------------------------------------------
def right_canonicalize(A: list) -> list:
    """Right isometries on sites 1..N-1 by QR of the transposed site matrices,
    the triangular factor absorbed into the left neighbour; site 0 normalised."""
    A = [a.copy() for a in A]
    N = len(A)
    for i in range(N - 1, 0, -1):
        chl, d, chr_ = A[i].shape
        M = A[i].reshape(chl, d * chr_)
        Q, Rm = np.linalg.qr(M.T)          # M^T = Q R  ->  M = R^T Q^T
        A[i] = Q.T.reshape(Q.shape[1], d, chr_)
        A[i - 1] = np.einsum("asm,mn->asn", A[i - 1], Rm.T, optimize=True)
    nrm = np.linalg.norm(A[0])
    if nrm > 0.0:  # a zero MPS has no normalised form and stays zero
        A[0] = A[0] / nrm
    return A


def left_isometry_error(A: np.ndarray) -> float:
    """max |sum_{a,s} A[a,s,c] A[a,s,c'] - delta_{cc'}|."""
    M = A.reshape(-1, A.shape[2])
    return float(np.max(np.abs(M.T @ M - np.eye(M.shape[1]))))


def right_isometry_error(A: np.ndarray) -> float:
    """max |sum_{s,c} A[a,s,c] A[a',s,c] - delta_{aa'}|."""
    M = A.reshape(A.shape[0], -1)
    return float(np.max(np.abs(M @ M.T - np.eye(M.shape[0]))))


def expectation(A: list, W: list) -> float:
    """<v, H v> by contracting the left environment through all sites (real
    for a Hermitian H: the real part is returned for complex tensors)."""
    L = np.ones((1, 1, 1))
    for a, w in zip(A, W):
        L = left_env(L, a, w)
    v = L.reshape(-1)[0]
    return float(v.real) if np.iscomplexobj(v) else float(v)


def overlap(A: list, B: list):
    """<v, w> by contracting the antilinear-form environment through all sites
    (a float for real tensors, a complex number for complex ones)."""
    F = np.ones((1, 1))
    for a, b in zip(A, B):
        F = left_env_linear(F, a, b)
    v = F.reshape(-1)[0]
    return complex(v) if np.iscomplexobj(v) else float(v)


# --------------------------------------------------------------------------
# local eigensolver: Lanczos with full re-orthogonalisation
# --------------------------------------------------------------------------
def lanczos_lowest(matvec, v0: np.ndarray, krylov_dim: int, breakdown_tol: float = 1e-14):
    """Lowest eigenpair of a symmetric operator in the Krylov space of v0.

    v_0 = v0/||v0||; for j = 0..k-1: w = H v_j, alpha_j = <v_j, w>,
    w -= alpha_j v_j + beta_{j-1} v_{j-1}, then w -= V (V^T w) twice (classical
    Gram-Schmidt, repeated), beta_j = ||w||; stop when
    beta_j <= breakdown_tol * max(1, |alpha_0|), else v_{j+1} = w / beta_j.
    The lowest eigenpair (lambda, y) of the tridiagonal T gives the Ritz
    vector sum_j y_j v_j, normalised.  Returns (lambda, vector, steps).
    """
    shape = v0.shape
    v = v0.reshape(-1) / np.linalg.norm(v0)
    n = v.size
    k = max(1, min(krylov_dim, n))
    V = np.zeros((k, n))
    V[0] = v
    alpha, beta = [], []
    for j in range(k):
        w = matvec(V[j].reshape(shape)).reshape(-1)
        a = float(V[j] @ w)
        alpha.append(a)
        w = w - a * V[j]
        if j > 0:
            w = w - beta[j - 1] * V[j - 1]
        for _ in range(2):
            w = w - V[: j + 1].T @ (V[: j + 1] @ w)
        b = float(np.linalg.norm(w))
        if j == k - 1 or b <= breakdown_tol * max(1.0, abs(alpha[0])):
            break
        beta.append(b)
        V[j + 1] = w / b
    m = len(alpha)
    T = np.diag(alpha) + np.diag(beta[: m - 1], 1) + np.diag(beta[: m - 1], -1)
    evals, evecs = np.linalg.eigh(T)
    y = evecs[:, 0]
    x = V[:m].T @ y
    x = x / np.linalg.norm(x)
    return float(evals[0]), x.reshape(shape), m


# --------------------------------------------------------------------------
# local linear solver: preconditioned conjugate gradients
# --------------------------------------------------------------------------
def pcg(matvec, b: np.ndarray, x0: np.ndarray, precond, rtol: float, maxiter: int):
    """Textbook PCG for an SPD operator: returns (x, relative residual, iterations).

    r = b - A x, z = P r, p = z; each step alpha = <r,z>/<p,Ap>, x += alpha p,
    r -= alpha Ap, stop when ||r|| <= rtol ||b||, z = P r,
    beta = <r_new, z_new>/<r, z>, p = z + beta p.
    """
    shape = b.shape
    bb = b.reshape(-1)
    x = x0.reshape(-1).copy()
    nb = float(np.linalg.norm(bb))
    if nb == 0.0:
        return np.zeros(shape), 0.0, 0
    r = bb - matvec(x.reshape(shape)).reshape(-1)
    rn = float(np.linalg.norm(r))
    if rn <= rtol * nb:
        return x.reshape(shape), rn / nb, 0
    z = precond(r)
    p = z.copy()
    rz = float(r @ z)
    it = 0
    for it in range(1, maxiter + 1):
        Ap = matvec(p.reshape(shape)).reshape(-1)
        alpha = rz / float(p @ Ap)
        x = x + alpha * p
        r = r - alpha * Ap
        rn = float(np.linalg.norm(r))
        if rn <= rtol * nb:
            break
        z = precond(r)
        rz_new = float(r @ z)
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x.reshape(shape), rn / nb, it


# --------------------------------------------------------------------------
# the sweep
# --------------------------------------------------------------------------
@dataclass
class SweepLog:
    energies: list = field(default_factory=list)       # one per half-sweep (last pair)
    bond_energies: list = field(default_factory=list)  # every local solve
    ranks: list = field(default_factory=list)          # per half-sweep: rank of each pair
    discarded: list = field(default_factory=list)      # per half-sweep: max discarded weight
    error: float = 0.0                                  # accumulated truncation bound (Sect. 2.3)
    local_iters: list = field(default_factory=list)


def _split(theta, chi_max, tol, mode, to_right: bool, normalize: bool):
    """Split a_n into the new A_n, A_{n+1}; the singular values go to the
    side the sweep moves toward (the next centre)."""
    chl, d1, d2, chr_ = theta.shape
    U, s, Vt, s_full, dw = svd_truncate(theta.reshape(chl * d1, d2 * chr_), chi_max, tol, mode)
    sig = s / np.linalg.norm(s) if normalize else s
    r = len(s)
    if to_right:
        A1 = U.reshape(chl, d1, r)
        A2 = (sig[:, None] * Vt).reshape(r, d2, chr_)
    else:
        A1 = (U * sig[None, :]).reshape(chl, d1, r)
        A2 = Vt.reshape(r, d2, chr_)
    return A1, A2, r, dw, s_full


def dmrg(W: list, A0: list, chi_max: int, tol: float, n_sweeps: int, krylov_dim: int,
         mode: str = TRUNC_WEIGHT, breakdown_tol: float = 1e-14):
    """Two-site DMRG (Sect. 3.1.1): minimise <v,Hv>/<v,v> pair by pair.

    With the centre on the active pair the norm matrix N_n is the identity, so
    the local problem H_n a = E N_n a is the standard symmetric eigenproblem.
    Returns (final energy, MPS, SweepLog).
    """
    N = len(A0)
    A = right_canonicalize(A0)
    Lenv = [None] * (N + 1)
    Renv = [None] * (N + 1)
    Lenv[0] = np.ones((1, 1, 1))
    Renv[N] = np.ones((1, 1, 1))
    for i in range(N - 1, 1, -1):
        Renv[i] = right_env(Renv[i + 1], A[i], W[i])
    log = SweepLog()
    E = None
    if N == 1:
        raise ValueError("two-site sweep needs N >= 2")
    for _ in range(n_sweeps):
        for direction in (+1, -1):
            pairs = range(0, N - 1) if direction > 0 else range(N - 2, -1, -1)
            ranks, dws = [], []
            for i in pairs:
                theta = two_site(A[i], A[i + 1])
                mv = lambda v, i=i: heff_apply(Lenv[i], W[i], W[i + 1], Renv[i + 2], v)
                E, theta, m = lanczos_lowest(mv, theta, krylov_dim, breakdown_tol)
                log.bond_energies.append(E)
                log.local_iters.append(m)
                A[i], A[i + 1], r, dw, _ = _split(theta, chi_max, tol, mode, direction > 0, True)
                ranks.append(r)
                dws.append(dw)
                log.error += dw
                if direction > 0:
                    Lenv[i + 1] = left_env(Lenv[i], A[i], W[i])
                else:
                    Renv[i + 1] = right_env(Renv[i + 2], A[i + 1], W[i + 1])
            log.energies.append(E)
            log.ranks.append(ranks)
            log.discarded.append(max(dws))
    return E, A, log


def dmrg_solve(W: list, B: list, X0: list, chi_max: int, tol: float, n_sweeps: int,
               pcg_rtol: float = 1e-12, pcg_maxiter: int = 500, mode: str = TRUNC_WEIGHT,
               precond: str = "jacobi", stop_rel_change: float = 0.0, extended: bool = False):
    """DMRG as a linear solver (Sect. 3.2.3): solve U x = b pair by pair.

    With x in mixed canonical form around the active pair, the local Galerkin
    system is U_n a_n = b_n with U_n the quadratic-form matrix of U and b_n the
    antilinear-form vector of b (Sect. 2.5).  Each local system is solved by
    PCG from the current a_n.  The split keeps the singular values
    unnormalised.  Returns (MPS, SweepLog with PCG iteration counts).

    extended = True carries the quadratic-form environments and the products
    U_n a in numpy's long double (a 64-bit significand on x86-64, 113 bits
    on aarch64) and rounds each product to FP64 once; everything else stays
    FP64.  Reading: the QTT Laplacian's MPO adds channels of size ~4^n that
    cancel to O(1) on smooth vectors, so FP64 environments alone bound the
    solution error near eps 4^n / 40; the wider environments lift that floor
    by the ratio of the two precisions.
    """
    xp = np.longdouble if extended else np.float64
    N = len(X0)
    A = right_canonicalize(X0)
    # undo the normalisation of the initial guess: keep its scale
    scale = np.sqrt(overlap(X0, X0))
    A[0] = A[0] * scale
    Lenv = [None] * (N + 1)
    Renv = [None] * (N + 1)
    Fenv = [None] * (N + 1)
    Genv = [None] * (N + 1)
    Lenv[0] = np.ones((1, 1, 1), dtype=xp)
    Renv[N] = np.ones((1, 1, 1), dtype=xp)
    Fenv[0] = np.ones((1, 1))
    Genv[N] = np.ones((1, 1))
    for i in range(N - 1, 1, -1):
        Renv[i] = right_env(Renv[i + 1], A[i], W[i])
        Genv[i] = right_env_linear(Genv[i + 1], A[i], B[i])
    log = SweepLog()
    prev = None
    for _ in range(n_sweeps):
        for direction in (+1, -1):
            pairs = range(0, N - 1) if direction > 0 else range(N - 2, -1, -1)
            ranks, dws = [], []
            for i in pairs:
                theta = two_site(A[i], A[i + 1])
                bvec = b_effective(Fenv[i], B[i], B[i + 1], Genv[i + 2])
                mv = lambda v, i=i: heff_apply(Lenv[i], W[i], W[i + 1], Renv[i + 2], v).astype(np.float64)
                if precond == "jacobi":
                    dg = heff_diagonal(Lenv[i], W[i], W[i + 1], Renv[i + 2]).reshape(-1).astype(np.float64)
                    pc = lambda r, dg=dg: r / dg
                else:
                    pc = lambda r: r
                theta, res, it = pcg(mv, bvec, theta, pc, pcg_rtol, pcg_maxiter)
                log.local_iters.append(it)
                A[i], A[i + 1], r, dw, _ = _split(theta, chi_max, tol, mode, direction > 0, False)
                ranks.append(r)
                dws.append(dw)
                log.error += dw
                if direction > 0:
                    Lenv[i + 1] = left_env(Lenv[i], A[i], W[i])
                    Fenv[i + 1] = left_env_linear(Fenv[i], A[i], B[i])
                else:
                    Renv[i + 1] = right_env(Renv[i + 2], A[i + 1], W[i + 1])
                    Genv[i + 1] = right_env_linear(Genv[i + 2], A[i + 1], B[i + 1])
            log.ranks.append(ranks)
            log.discarded.append(max(dws))
        if stop_rel_change > 0.0:
            cur = [a.copy() for a in A]
            if prev is not None:
                d2 = overlap(cur, cur) + overlap(prev, prev) - 2.0 * overlap(cur, prev)
                if np.sqrt(max(d2, 0.0)) <= stop_rel_change * np.sqrt(overlap(cur, cur)):
                    break
            prev = cur
    return A, log


# --------------------------------------------------------------------------
# variational compression (Sect. 2.3; eq. of psi_opt and the join of sums, Sect. 2.4.1)
# --------------------------------------------------------------------------
def distance2(A: list, B: list) -> float:
    """|A - B|^2 from three overlaps (Sect. 2.5's forms)."""
    return overlap(A, A) + overlap(B, B) - 2.0 * overlap(A, B)


def simplify(B: list, X0: list, chi_max: int, tol: float, n_sweeps: int, mode: str = TRUNC_WEIGHT):
    """The MPS x of bond dimension <= chi_max closest to b, by two-site sweeps.

    With x in mixed canonical form around the active pair, |x - b|^2 equals
    a^T a - 2 a^T b_n + |b|^2 (the quadratic form of Sect. 2.5 has the identity
    as its matrix), so the best pair tensor is a_n = b_n, the antilinear-form
    vector of b; it is split by the truncated SVD with the singular values
    kept unnormalised, and the sweep moves on.  Sums of MPS are compressed by
    passing their direct sum as b.  Starts from the guess X0 (brought to
    right-canonical form).  Returns (MPS, SweepLog).
    """
    N = len(X0)
    A = right_canonicalize(X0)
    Fenv = [None] * (N + 1)
    Genv = [None] * (N + 1)
    Fenv[0] = np.ones((1, 1))
    Genv[N] = np.ones((1, 1))
    for i in range(N - 1, 1, -1):
        Genv[i] = right_env_linear(Genv[i + 1], A[i], B[i])
    log = SweepLog()
    for _ in range(n_sweeps):
        for direction in (+1, -1):
            pairs = range(0, N - 1) if direction > 0 else range(N - 2, -1, -1)
            ranks, dws = [], []
            for i in pairs:
                theta = b_effective(Fenv[i], B[i], B[i + 1], Genv[i + 2])
                A[i], A[i + 1], r, dw, _ = _split(theta, chi_max, tol, mode, direction > 0, False)
                ranks.append(r)
                dws.append(dw)
                log.error += dw
                if direction > 0:
                    Fenv[i + 1] = left_env_linear(Fenv[i], A[i], B[i])
                else:
                    Genv[i + 1] = right_env_linear(Genv[i + 2], A[i + 1], B[i + 1])
            log.ranks.append(ranks)
            log.discarded.append(max(dws))
    return A, log


# --------------------------------------------------------------------------
# MPO times MPS (Sect. 2.4.2, matrix-vector product): exact and variational
# --------------------------------------------------------------------------
def mpo_mps_product(W: list, B: list) -> list:
    """The exact product U v as an MPS with enlarged tensors (Sect. 2.4.2, eq. of
    C): C[(beta, alpha), j, (beta', alpha')] = sum_i W[beta, j, i, beta'] B[alpha, i, alpha'],
    the MPO bond running slower than the MPS bond in the combined index."""
    C = []
    for Wn, Bn in zip(W, B):
        T = np.einsum("bjif,aic->bajfc", Wn, Bn, optimize=True)
        Db, Da, d, Df, Dc = T.shape
        C.append(T.reshape(Db * Da, d, Df * Dc))
    return C


def left_env_mixed(L: np.ndarray, X: np.ndarray, W: np.ndarray, B: np.ndarray) -> np.ndarray:
    """The left environment of <x, U b> (Sect. 2.5 with different bra and ket):
    L_{n+1}[c', f, c] = sum conj(X[a', s', c']) L_n[a', b, a] W[b, s', s, f] B[a, s, c],
    L[a', b, a] with a' a bond of x and a a bond of b."""
    T = np.einsum("pbq,qsc->pbsc", L, B, optimize=True)  # T[a', b, s, c]
    T = np.einsum("pbsc,bjsf->pjcf", T, W, optimize=True)  # T[a', s', c, f]
    return np.einsum("pjcf,pjr->rfc", T, X.conj(), optimize=True)


def right_env_mixed(R: np.ndarray, X: np.ndarray, W: np.ndarray, B: np.ndarray) -> np.ndarray:
    """R_n[a', b, a] = sum conj(X[a', s', c']) W[b, s', s, f] R_{n+1}[c', f, c] B[a, s, c]."""
    T = np.einsum("rfc,qsc->rfqs", R, B, optimize=True)  # T[c', f, a, s]
    T = np.einsum("rfqs,bjsf->rqbj", T, W, optimize=True)  # T[c', a, b, s']
    return np.einsum("rqbj,pjr->pbq", T, X.conj(), optimize=True)


def apply_mpo(W: list, B: list, X0: list, chi_max: int, tol: float, n_sweeps: int,
              mode: str = TRUNC_WEIGHT):
    """The MPS x of bond dimension <= chi_max closest to U b (Sect. 2.4.2, the
    variational matrix-vector product), by two-site sweeps.

    With x in mixed canonical form around the active pair,
    |x - U b|^2 = a^T a - 2 a^T (U b)_n + |U b|^2, so the best pair tensor is
    (U b)_n = L_n W_n W_{n+1} R_{n+2} applied to b's two-site tensor, the
    environments being those of <x, U b>; it is split with the singular
    values kept unnormalised, and the sweep moves on.  The enlarged product
    of eq. C is never formed.  Starts from the guess X0 (brought to
    right-canonical form).  Returns (MPS, SweepLog).
    """
    N = len(X0)
    A = right_canonicalize(X0)
    Lenv = [None] * (N + 1)
    Renv = [None] * (N + 1)
    Lenv[0] = np.ones((1, 1, 1))
    Renv[N] = np.ones((1, 1, 1))
    for i in range(N - 1, 1, -1):
        Renv[i] = right_env_mixed(Renv[i + 1], A[i], W[i], B[i])
    log = SweepLog()
    for _ in range(n_sweeps):
        for direction in (+1, -1):
            pairs = range(0, N - 1) if direction > 0 else range(N - 2, -1, -1)
            ranks, dws = [], []
            for i in pairs:
                theta = heff_apply(Lenv[i], W[i], W[i + 1], Renv[i + 2], two_site(B[i], B[i + 1]))
                A[i], A[i + 1], r, dw, _ = _split(theta, chi_max, tol, mode, direction > 0, False)
                ranks.append(r)
                dws.append(dw)
                log.error += dw
                if direction > 0:
                    Lenv[i + 1] = left_env_mixed(Lenv[i], A[i], W[i], B[i])
                else:
                    Renv[i + 1] = right_env_mixed(Renv[i + 2], A[i + 1], W[i + 1], B[i + 1])
            log.ranks.append(ranks)
            log.discarded.append(max(dws))
    return A, log


# --------------------------------------------------------------------------
# global conjugate gradients on MPS (Sect. 3.2.1, CGS; Fig. cgs)
# --------------------------------------------------------------------------
def mps_sum(weights: list, states: list) -> list:
    """The joined MPS of sum_l w_l psi_l (Sect. 2.4.1, join): the first site a
    row of the terms' tensors (each scaled by its weight), the last site a
    column, the sites between block diagonal."""
    N = len(states[0])
    out = []
    for n in range(N):
        ts = [st[n] for st in states]
        if n == 0:
            ts = [w * t for w, t in zip(weights, ts)]
        if N == 1:
            out.append(sum(ts))
        elif n == 0:
            out.append(np.concatenate(ts, axis=2))
        elif n == N - 1:
            out.append(np.concatenate(ts, axis=0))
        else:
            rows = sum(t.shape[0] for t in ts)
            cols = sum(t.shape[2] for t in ts)
            C = np.zeros((rows, ts[0].shape[1], cols))
            r0 = c0 = 0
            for t in ts:
                C[r0:r0 + t.shape[0], :, c0:c0 + t.shape[2]] = t
                r0 += t.shape[0]
                c0 += t.shape[2]
            out.append(C)
    return out


def cgs_solve(W: list, B: list, X0: list, chi_max: int, tol: float, rtol: float, maxiter: int,
              n_sweeps: int = 2, mode: str = TRUNC_WEIGHT):
    """Conjugate gradients for the symmetric MPO U (= W) and MPS b, in the
    order of Fig. cgs: x = simplify(guess); r = b - U x; p = r; then per step
    alpha = |r|^2 / <p, U p>, x = simplify(x + alpha p), r = b - U x,
    beta = (|r_new| / |r_old|)^2, p = simplify(r + beta p).

    Readings where the printed listing departs from the standard recurrence
    the paper cites: with r = b - U x the step is x + alpha p (the listing
    prints x - a p); beta is the ratio of the squared residual norms (the
    listing omits the square).  And the residual b - U x is compressed,
    r = simplify(b - U x), before its norm is taken: the norm of the lazy sum
    from <b,b> - 2<b,Ux> + <Ux,Ux> cannot resolve |r| below ~1e-8 |b| in FP64.
    Every compression is the variational simplify (U x the variational
    MPO-MPS product) with n_sweeps sweeps, started from the previous value of
    the same MPS.  Stops when |r| < rtol |b|, when |r| = 0, or after maxiter
    steps.  Returns (x, |r|, steps, residual history).
    """
    nb = float(np.sqrt(overlap(B, B)))
    x, _ = simplify(X0, X0, chi_max, tol, n_sweeps, mode)
    y, _ = apply_mpo(W, x, x, chi_max, tol, n_sweeps, mode)
    r, _ = simplify(mps_sum([1.0, -1.0], [B, y]), y, chi_max, tol, n_sweeps, mode)
    res = float(np.sqrt(overlap(r, r)))
    p = [t.copy() for t in r]
    hist = [res]
    steps = 0
    while steps < maxiter and not res < rtol * nb and res > 0.0:  # |r| = 0 is convergence
        alpha = res * res / expectation(p, W)
        x, _ = simplify(mps_sum([1.0, alpha], [x, p]), x, chi_max, tol, n_sweeps, mode)
        y, _ = apply_mpo(W, x, y, chi_max, tol, n_sweeps, mode)
        r, _ = simplify(mps_sum([1.0, -1.0], [B, y]), r, chi_max, tol, n_sweeps, mode)
        res_new = float(np.sqrt(overlap(r, r)))
        beta = (res_new / res) ** 2
        p, _ = simplify(mps_sum([1.0, beta], [r, p]), p, chi_max, tol, n_sweeps, mode)
        res = res_new
        hist.append(res)
        steps += 1
    return x, res, steps, hist


# --------------------------------------------------------------------------
# two-site TDVP (Sect. 7.3, TDVP) for the real generator L = -H
# --------------------------------------------------------------------------
def heff1_apply(L, W, R, A) -> np.ndarray:
    """One-site effective operator:
    (H^(n) a)[a', s', c'] = sum L[a', b, a] W[b, s', s, f] R[c', f, c] a[a, s, c],
    as three pairwise index sums (over a, over (b, s), over (c, f))."""
    T = np.einsum("pbq,qsc->pbsc", L, A, optimize=True)  # T[a', b, s, c]
    T = np.einsum("pbsc,bjsf->pjcf", T, W, optimize=True)  # T[a', s', c, f]
    return np.einsum("pjcf,rfc->pjr", T, R, optimize=True)  # y[a', s', c']


def krylov_expm(matvec, v0: np.ndarray, tau, krylov_dim: int, breakdown_tol: float = 1e-14):
    """exp(tau H) v0 for Hermitian H, in the Krylov space of v0.

    The Lanczos recurrence of lanczos_lowest (full re-orthogonalisation)
    gives the orthonormal basis V and the real tridiagonal T = V^H H V; then
    exp(tau H) v0 ~ |v0| V exp(tau T) e_1 with exp(tau T) = Q exp(tau Lambda) Q^T
    from the eigendecomposition of T.  tau is real (imaginary time) or
    imaginary (real time, tau = -i dt); with a complex v0 or tau the basis is
    complex and every inner product conjugates its first argument.  Returns
    (vector, steps, <v0,H v0>/<v0,v0>).
    """
    shape = v0.shape
    cplx = np.iscomplexobj(v0) or np.iscomplexobj(tau)
    nrm = float(np.linalg.norm(v0))
    v = v0.reshape(-1) / nrm
    n = v.size
    k = max(1, min(krylov_dim, n))
    V = np.zeros((k, n), dtype=complex if cplx else float)
    V[0] = v
    alpha, beta = [], []
    for j in range(k):
        w = matvec(V[j].reshape(shape)).reshape(-1)
        a = float(np.vdot(V[j], w).real) if cplx else float(V[j] @ w)
        alpha.append(a)
        w = w - a * V[j]
        if j > 0:
            w = w - beta[j - 1] * V[j - 1]
        for _ in range(2):
            if cplx:
                w = w - V[: j + 1].T @ (V[: j + 1].conj() @ w)
            else:
                w = w - V[: j + 1].T @ (V[: j + 1] @ w)
        b = float(np.linalg.norm(w))
        if j == k - 1 or b <= breakdown_tol * max(1.0, abs(alpha[0])):
            break
        beta.append(b)
        V[j + 1] = w / b
    m = len(alpha)
    T = np.diag(alpha) + np.diag(beta[: m - 1], 1) + np.diag(beta[: m - 1], -1)
    lam, Q = np.linalg.eigh(T)
    c = Q @ (np.exp(tau * lam) * Q[0, :])
    x = nrm * (V[:m].T @ c)
    return x.reshape(shape), m, alpha[0]


def tdvp(W: list, A0: list, dt: float, n_steps: int, chi_max: int, tol: float, krylov_dim: int,
         mode: str = TRUNC_WEIGHT, breakdown_tol: float = 1e-14, real_time: bool = False):
    """Two-site TDVP for the generator L = -H (imaginary time), normalised, or
    with real_time for L = -i H (the Schroedinger equation; complex tensors).

    One time step is a left-to-right then a right-to-left sweep (the
    symmetric second-order integrator).  At bond (n, n+1): the pair tensor
    evolves forward, a <- exp(dt/2 L_(n,n+1)) a; the truncated SVD splits it
    with the singular values normalised; unless the bond is the last of the
    half sweep, the site that now holds the centre evolves backward with its
    one-site operator, A <- exp(-dt/2 L_(site)) A, and is normalised (real
    time preserves the norm; the normalisation only removes the truncation's
    and the Krylov space's loss).  Returns (<psi|H|psi> / <psi|psi>, MPS, SweepLog).
    """
    N = len(A0)
    if N < 2:
        raise ValueError("two-site TDVP needs N >= 2")
    fwd, bwd = (-0.5j * dt, 0.5j * dt) if real_time else (-0.5 * dt, 0.5 * dt)
    A = right_canonicalize([a.astype(complex) for a in A0] if real_time else A0)
    Lenv = [None] * (N + 1)
    Renv = [None] * (N + 1)
    Lenv[0] = np.ones((1, 1, 1))
    Renv[N] = np.ones((1, 1, 1))
    for i in range(N - 1, 1, -1):
        Renv[i] = right_env(Renv[i + 1], A[i], W[i])
    log = SweepLog()
    for _ in range(n_steps):
        for direction in (+1, -1):
            pairs = range(0, N - 1) if direction > 0 else range(N - 2, -1, -1)
            ranks, dws = [], []
            for i in pairs:
                theta = two_site(A[i], A[i + 1])
                mv2 = lambda v, i=i: heff_apply(Lenv[i], W[i], W[i + 1], Renv[i + 2], v)
                theta, m, _ = krylov_expm(mv2, theta, fwd, krylov_dim, breakdown_tol)
                log.local_iters.append(m)
                A[i], A[i + 1], r, dw, _ = _split(theta, chi_max, tol, mode, direction > 0, True)
                ranks.append(r)
                dws.append(dw)
                log.error += dw
                if direction > 0:
                    Lenv[i + 1] = left_env(Lenv[i], A[i], W[i])
                    if i < N - 2:
                        mv1 = lambda v, i=i: heff1_apply(Lenv[i + 1], W[i + 1], Renv[i + 2], v)
                        a, _, _ = krylov_expm(mv1, A[i + 1], bwd, krylov_dim, breakdown_tol)
                        A[i + 1] = a / np.linalg.norm(a)
                else:
                    Renv[i + 1] = right_env(Renv[i + 2], A[i + 1], W[i + 1])
                    if i > 0:
                        mv1 = lambda v, i=i: heff1_apply(Lenv[i], W[i], Renv[i + 1], v)
                        a, _, _ = krylov_expm(mv1, A[i], bwd, krylov_dim, breakdown_tol)
                        A[i] = a / np.linalg.norm(a)
            log.ranks.append(ranks)
            log.discarded.append(max(dws))
    nn = overlap(A, A)
    E = expectation(A, W) / (nn.real if isinstance(nn, complex) else nn)
    log.energies.append(E)
    return E, A, log

