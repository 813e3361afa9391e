"""Section 2.4: the discrete integral system (Definition 4, Theorem 1, Remark 1).

Test infrastructure: see the package docstring.

Trace unknowns are ordered by interface: interface i (between 0-based layers
i and i+1) carries trace 2i = u^i_{n} (= u^{i+1}_0) and trace 2i+1 =
u^i_{n+1} (= u^{i+1}_1), each a vector of n_t complex values.  Rows follow the
printed M: row 2i is the GRF of layer i at j = n, row 2i+1 that of layer i+1
at j = 1; for M_0 (Remark 1) row 2i is layer i at j = n+1 and row 2i+1 is
layer i+1 at j = 0.
"""
from __future__ import annotations

import numpy as np


def down_terms(G: dict, j: int, h: float, cols) -> list:
    """Matrix form of the down-going incomplete integral (Section 2.3):
    G_down_j(v_0, v_1) = (1/h) [G(z_j, z_1)  -G(z_j, z_0)] (v_0; v_1).
    ``cols`` are the unknowns holding (v_0, v_1)."""
    return [(cols[0], G[(j, 1)] / h), (cols[1], -G[(j, 0)] / h)]


def up_terms(G: dict, j: int, n: int, h: float, cols) -> list:
    """Matrix form of the up-going incomplete integral (Section 2.3):
    G_up_j(v_n, v_{n+1}) = (1/h) [-G(z_j, z_{n+1})  G(z_j, z_n)] (v_n; v_{n+1})."""
    return [(cols[0], -G[(j, n + 1)] / h), (cols[1], G[(j, n)] / h)]


class BlockSystem:
    """A square block-sparse operator given row by row as lists of
    (column, block) terms; a block is an n_t x n_t array or the scalar -1
    standing for minus the identity (the paper's (1/h) I with (I v)_i = h v_i)."""

    def __init__(self, nrows: int, ncols: int, nt: int):
        self.nrows, self.ncols, self.nt = nrows, ncols, nt
        self.rows = [[] for _ in range(nrows)]

    def add(self, row: int, terms) -> None:
        self.rows[row].extend(terms)

    def apply(self, x: np.ndarray, row_filter=None) -> np.ndarray:
        """y = A x, x of shape (ncols * n_t,); ``row_filter(row, col)`` keeps a subset of terms."""
        nt = self.nt
        X = x.reshape(self.ncols, nt)
        Y = np.zeros((self.nrows, nt), dtype=np.complex128)
        for r, terms in enumerate(self.rows):
            for c, B in terms:
                if row_filter is not None and not row_filter(r, c):
                    continue
                Y[r] += (-X[c]) if np.isscalar(B) else B @ X[c]
        return Y.reshape(-1)

    def dense(self, row_filter=None) -> np.ndarray:
        nt = self.nt
        A = np.zeros((self.nrows * nt, self.ncols * nt), dtype=np.complex128)
        eye = np.eye(nt)
        for r, terms in enumerate(self.rows):
            for c, B in terms:
                if row_filter is not None and not row_filter(r, c):
                    continue
                A[r * nt : (r + 1) * nt, c * nt : (c + 1) * nt] += -eye if np.isscalar(B) else B
        return A


def _top(l: int):
    """Unknowns (u_0, u_1) of layer l: the traces of interface l-1."""
    return (2 * (l - 1), 2 * (l - 1) + 1)


def _bot(l: int):
    """Unknowns (u_n, u_{n+1}) of layer l: the traces of interface l."""
    return (2 * l, 2 * l + 1)


def integral_system(blocks: list, ns: list, h: float, nt: int) -> BlockSystem:
    """M of Definition 4: the GRF of Lemma 1 evaluated at j = 1 and j = n of
    every layer, with the unknown trace moved to the left-hand side."""
    L = len(blocks)
    S = BlockSystem(2 * (L - 1), 2 * (L - 1), nt)
    for l in range(L):
        G, n = blocks[l], ns[l]
        for j, row, ident in ((n, 2 * l, 2 * l), (1, 2 * l - 1, 2 * l - 1)):
            if (j == n and l == L - 1) or (j == 1 and l == 0):
                continue
            terms = []
            if l > 0:
                terms += down_terms(G, j, h, _top(l))
            if l < L - 1:
                terms += up_terms(G, j, n, h, _bot(l))
            terms.append((ident, -1))
            S.add(row, terms)
    return S


def integral_system_outside(blocks: list, ns: list, h: float, nt: int) -> BlockSystem:
    """M_0 of Remark 1: the GRF at j = n+1 and j = 0, where Lemma 2 makes the
    field vanish (no identity blocks)."""
    L = len(blocks)
    S = BlockSystem(2 * (L - 1), 2 * (L - 1), nt)
    for l in range(L):
        G, n = blocks[l], ns[l]
        for j, row in ((n + 1, 2 * l), (0, 2 * l - 1)):
            if (j == n + 1 and l == L - 1) or (j == 0 and l == 0):
                continue
            terms = []
            if l > 0:
                terms += down_terms(G, j, h, _top(l))
            if l < L - 1:
                terms += up_terms(G, j, n, h, _bot(l))
            S.add(row, terms)
    return S


def integral_rhs(newton: list, ns: list, nt: int, outside: bool = False) -> np.ndarray:
    """f (Eq. of Definition 4) or f_0 (Remark 1): local Newton potentials at the
    trace rows, stacked in row order.  ``newton[l]`` maps a paper row index j
    to N^l_j f^l (a length n_t vector)."""
    L = len(newton)
    out = np.zeros((2 * (L - 1), nt), dtype=np.complex128)
    for i in range(L - 1):
        n_up = ns[i]
        if outside:
            out[2 * i] = newton[i][n_up + 1]
            out[2 * i + 1] = newton[i + 1][0]
        else:
            out[2 * i] = newton[i][n_up]
            out[2 * i + 1] = newton[i + 1][1]
    return out.reshape(-1)
