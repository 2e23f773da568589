"""Operator inputs of the sweep: MPO tensors for the models the workloads use.

Every MPO is a list of real float64 arrays W[n] with shape (D_l, d, d, D_r),
indexed W[n][b, j, i, f] with j the output (row) and i the input (column)
physical index, the storage order of Sect. 2.2 (matrix representation).  The
first tensor has D_l = 1 and the last D_r = 1, the open boundary of Sect. 2.1.

These builders describe the problem (the Hamiltonian or the discretised
operator); they are inputs, not steps of the sweep.  The tests pin every one
of them against a dense Kronecker-product construction.

Finite-state-machine form.  A sum of products of one-site operators is written
with bond states: state 0 means "nothing placed yet" (identity to the left),
the last state means "term complete" (identity to the right) and the middle
states carry a half-placed term across the bond.
"""
from __future__ import annotations

import numpy as np

PAULI_X = np.array([[0.0, 1.0], [1.0, 0.0]])
PAULI_Z = np.array([[1.0, 0.0], [0.0, -1.0]])
ID2 = np.eye(2)
# sigma^+ = |0><1| and sigma^- = |1><0|; X X + Y Y = 2 (s+ s- + s- s+) keeps
# the XXZ operator real.
SIGMA_P = np.array([[0.0, 1.0], [0.0, 0.0]])
SIGMA_M = np.array([[0.0, 0.0], [1.0, 0.0]])


def _open_chain(bulk: np.ndarray, n: int) -> list:
    """Open chain from one bulk tensor: first row on site 0, last column on site n-1."""
    out = []
    for i in range(n):
        W = bulk.copy()
        if i == 0:
            W = W[0:1]
        if i == n - 1:
            W = W[..., -1:]
        out.append(W)
    return out


def tfim(n: int, g: float) -> list:
    """Open transverse-field Ising chain H = -sum Z_i Z_{i+1} - g sum X_i (Pauli), D = 3."""
    W = np.zeros((3, 2, 2, 3))
    W[0, :, :, 0] = ID2
    W[0, :, :, 1] = -PAULI_Z
    W[0, :, :, 2] = -g * PAULI_X
    W[1, :, :, 2] = PAULI_Z
    W[2, :, :, 2] = ID2
    return _open_chain(W, n)


def xxz(n: int, delta: float) -> list:
    """Open XXZ chain H = sum (X X + Y Y + delta Z Z) on neighbours (Pauli), D = 5."""
    W = np.zeros((5, 2, 2, 5))
    W[0, :, :, 0] = ID2
    W[0, :, :, 1] = 2.0 * SIGMA_P
    W[0, :, :, 2] = 2.0 * SIGMA_M
    W[0, :, :, 3] = delta * PAULI_Z
    W[1, :, :, 4] = SIGMA_M
    W[2, :, :, 4] = SIGMA_P
    W[3, :, :, 4] = PAULI_Z
    W[4, :, :, 4] = ID2
    return _open_chain(W, n)


def heisenberg_graph(n: int, bonds: list) -> list:
    """H = sum_{(i,j,J)} J (X_i X_j + Y_i Y_j + Z_i Z_j), i < j, any range.

    Bond states across the cut between sites k and k+1: 0 (nothing placed),
    one state per (open site i <= k, operator in {s+, s-, Z}) for every i that
    still has a partner j > k, and the final "complete" state.  This is the
    exact (uncompressed) finite-state-machine MPO of Sect. 8.1's interaction
    graph; its bond dimension is 2 + 3 * (number of open sites).
    """
    J = {}
    for (i, j, c) in bonds:
        if i == j:
            raise ValueError("self interaction")
        a, b = min(i, j), max(i, j)
        J[(a, b)] = J.get((a, b), 0.0) + float(c)
    ops_first = [2.0 * SIGMA_P, 2.0 * SIGMA_M, PAULI_Z]
    ops_second = [SIGMA_M, SIGMA_P, PAULI_Z]
    # open[k] = sorted sites i <= k with a partner j > k (cut after site k)
    open_sites = []
    for k in range(n):
        open_sites.append(sorted({a for (a, b) in J if a <= k < b}))

    def states(k):  # bond to the right of site k
        if k < 0 or k >= n - 1:
            return None
        return open_sites[k]

    out = []
    for k in range(n):
        left = states(k - 1)
        right = states(k)
        Dl = 1 if left is None else 2 + 3 * len(left)
        Dr = 1 if right is None else 2 + 3 * len(right)
        W = np.zeros((Dl, 2, 2, Dr))
        # index helpers
        def lidx(tag, i=None, a=None):
            if left is None:
                return 0 if tag == "start" else None
            if tag == "start":
                return 0
            if tag == "done":
                return Dl - 1
            return 1 + 3 * left.index(i) + a

        def ridx(tag, i=None, a=None):
            if right is None:
                return 0 if tag == "done" else None
            if tag == "start":
                return 0
            if tag == "done":
                return Dr - 1
            return 1 + 3 * right.index(i) + a

        # start -> start (identity), done -> done (identity)
        ls, rs = lidx("start"), ridx("start")
        if ls is not None and rs is not None:
            W[ls, :, :, rs] += ID2
        ld, rd = lidx("done"), ridx("done")
        if ld is not None and rd is not None and left is not None:
            W[ld, :, :, rd] += ID2
        # open a new term at site k
        if ls is not None and right is not None and k in right:
            for a in range(3):
                W[ls, :, :, ridx("open", k, a)] += ops_first[a]
        # carry open terms through site k, or close them at site k
        if left is not None:
            for i in left:
                for a in range(3):
                    li = lidx("open", i, a)
                    c = J.get((i, k), 0.0)
                    if c != 0.0 and rd is not None:
                        W[li, :, :, rd] += c * ops_second[a]
                    if right is not None and i in right:
                        W[li, :, :, ridx("open", i, a)] += ID2
        out.append(W)
    return out


def j1j2_cylinder_bonds(width: int, length: int, j1: float, j2: float) -> list:
    """Bonds of the J1-J2 model on a width x length cylinder, site = width*x + y.

    Periodic in y, open in x.  J1 on nearest neighbours, J2 on both diagonals
    of every plaquette (including those that wrap around y).
    """
    bonds = {}

    def add(a, b, c):
        key = (min(a, b), max(a, b))
        bonds[key] = bonds.get(key, 0.0) + c

    def site(x, y):
        return width * x + (y % width)

    for x in range(length):
        for y in range(width):
            if width > 2 or y + 1 < width:
                add(site(x, y), site(x, y + 1), j1)
            if x + 1 < length:
                add(site(x, y), site(x + 1, y), j1)
                if j2 != 0.0:
                    add(site(x, y), site(x + 1, y + 1), j2)
                    add(site(x, y), site(x + 1, y - 1), j2)
    return [(a, b, c) for (a, b), c in sorted(bonds.items())]


def laplacian_qtt_1d(n: int, h: float) -> list:
    """(2 I - S+ - S-)/h^2 on 2^n interior nodes, MSB-first qubits, zero fill.

    (S+ v)_i = v_{i+1} and (S- v)_i = v_{i-1}, zero outside [0, 2^n): the
    open-boundary displacements of Sect. 5.1.  Bond states carry the pending
    carry of the binary increment (1) or decrement (2) from the least
    significant qubit (last site) toward the most significant one; state 0
    means no pending carry.  A carry out of the first site is dropped, which
    is exactly the zero fill.  D = 3.
    """
    c = 1.0 / (h * h)
    W = np.zeros((3, 2, 2, 3))
    # f = 0: no carry from the right -> identity, b = 0
    W[0, 0, 0, 0] = 1.0
    W[0, 1, 1, 0] = 1.0
    # f = 1: increment, input = output + carry
    W[0, 0, 1, 1] = 1.0  # j=0 -> i=1, carry absorbed
    W[1, 1, 0, 1] = 1.0  # j=1 -> i=0, carry continues
    # f = 2: decrement, input = output - borrow
    W[0, 1, 0, 2] = 1.0  # j=1 -> i=0, borrow absorbed
    W[2, 0, 1, 2] = 1.0  # j=0 -> i=1, borrow continues
    right = np.array([2.0 * c, -c, -c])
    out = []
    for k in range(n):
        Wk = W.copy()
        if k == 0:
            Wk = Wk[0:1]
        if k == n - 1:
            Wk = np.einsum("bjif,f->bji", Wk, right)[..., None]
        out.append(Wk)
    return out


def laplacian_qtt_2d(n: int, h: float) -> list:
    """-Laplacian on a 2^n x 2^n interior grid, interleaved order B, D = 5.

    Sites alternate x_1, y_1, x_2, y_2, ..., x_n, y_n (most significant bit
    first, Sect. 4.1 order "B").  The operator is A_x (x) I + I (x) A_y with
    A = (2 I - S+ - S-)/h^2.  Bond states: 0 no pending carry, 1/2 pending
    x increment/decrement, 3/4 pending y increment/decrement.  A site of one
    coordinate passes the other coordinate's pending carry through with the
    identity.  The right boundary vector weights the states by
    (4, -1, -1, -1, -1)/h^2.
    """
    c = 1.0 / (h * h)

    def site_tensor(is_x: bool) -> np.ndarray:
        W = np.zeros((5, 2, 2, 5))
        W[0, 0, 0, 0] = W[0, 1, 1, 0] = 1.0
        own = (1, 2) if is_x else (3, 4)
        other = (3, 4) if is_x else (1, 2)
        inc, dec = own
        W[0, 0, 1, inc] = 1.0
        W[inc, 1, 0, inc] = 1.0
        W[0, 1, 0, dec] = 1.0
        W[dec, 0, 1, dec] = 1.0
        for s in other:
            W[s, 0, 0, s] = W[s, 1, 1, s] = 1.0
        return W

    right = np.array([4.0 * c, -c, -c, -c, -c])
    out = []
    L = 2 * n
    for k in range(L):
        Wk = site_tensor(k % 2 == 0)
        if k == 0:
            Wk = Wk[0:1]
        if k == L - 1:
            Wk = np.einsum("bjif,f->bji", Wk, right)[..., None]
        out.append(Wk)
    return out


def identity_mpo(n: int, d: int = 2) -> list:
    return [np.eye(d).reshape(1, d, d, 1).copy() for _ in range(n)]
