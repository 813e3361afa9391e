"""Section 3 (polarized traces) and Section 4.1 (Gauss-Seidel), as the paper defines them.

Test infrastructure: see the package docstring.

Unknowns of the polarized system (Definition 9) are (u_down, u_up), each
ordered like the traces of the integral system: column c < 2(L-1) is the
down-going part of trace c, column 2(L-1) + c its up-going part.  Rows follow
Definition 9: the first 2(L-1) rows are the M-rows (layer i at j = n, layer
i+1 at j = 1), the next 2(L-1) the M_0-rows (layer i at j = n+1, layer i+1
at j = 0).

The blocks are assembled from the four scalar jump-condition equations of
Section 3.5 and the matrix form of Definition 2, not from the printed block
matrices, which carry misprints.  In those equations the terms that the
annihilation relations (Definition 5) remove are G_down_1(u_up) and
G_up_n(u_down); the terms G_down_0(u_up) = -u_up_0 and G_up_{n+1}(u_down) =
-u_down_{n+1} (Lemma 6 with Lemma 4) are moved to the right-hand side.
Reading: the right-hand side of the fourth equation is u_down_{n+1} (printed
as u_down_n); this is what the jump relation of Lemma 4 gives and what the
proof of Lemma 6 uses.
"""
from __future__ import annotations

import numpy as np

from .integral import BlockSystem, _bot, _top, down_terms, up_terms


def polarized_jump_system(blocks: list, ns: list, h: float, nt: int) -> BlockSystem:
    """The polarized system completed with jump conditions (Definition 9)."""
    L = len(blocks)
    T = 2 * (L - 1)  # traces
    S = BlockSystem(2 * T, 2 * T, nt)
    dn = lambda cols: tuple(c for c in cols)  # noqa: E731  (down-going columns)
    up = lambda cols: tuple(T + c for c in cols)  # noqa: E731  (up-going columns)

    for l in range(L):
        G, n = blocks[l], ns[l]
        has_top, has_bot = l > 0, l < L - 1
        if has_bot:
            # (jump 2) j = n:  G_down_n(u_up + u_down) + G_up_n(u_up) = u_up_n + u_down_n - N_n f
            terms = []
            if has_top:
                terms += down_terms(G, n, h, up(_top(l))) + down_terms(G, n, h, dn(_top(l)))
            terms += up_terms(G, n, n, h, up(_bot(l)))
            terms += [(T + 2 * l, -1), (2 * l, -1)]
            S.add(2 * l, terms)
            # (jump 4) j = n+1:  G_down_{n+1}(u_up + u_down) + G_up_{n+1}(u_up) = u_down_{n+1} - N_{n+1} f
            terms = []
            if has_top:
                terms += down_terms(G, n + 1, h, up(_top(l))) + down_terms(G, n + 1, h, dn(_top(l)))
            terms += up_terms(G, n + 1, n, h, up(_bot(l)))
            terms += [(2 * l + 1, -1)]
            S.add(T + 2 * l, terms)
        if has_top:
            # (jump 1) j = 1:  G_up_1(u_up + u_down) + G_down_1(u_down) = u_up_1 + u_down_1 - N_1 f
            terms = []
            if has_bot:
                terms += up_terms(G, 1, n, h, up(_bot(l))) + up_terms(G, 1, n, h, dn(_bot(l)))
            terms += down_terms(G, 1, h, dn(_top(l)))
            terms += [(T + 2 * l - 1, -1), (2 * l - 1, -1)]
            S.add(2 * l - 1, terms)
            # (jump 3) j = 0:  G_up_0(u_up + u_down) + G_down_0(u_down) = u_up_0 - N_0 f
            terms = []
            if has_bot:
                terms += up_terms(G, 0, n, h, up(_bot(l))) + up_terms(G, 0, n, h, dn(_bot(l)))
            terms += down_terms(G, 0, h, dn(_top(l)))
            terms += [(T + 2 * l - 2, -1)]
            S.add(T + 2 * l - 1, terms)
    return S


def polarized_rhs(f_under: np.ndarray, f0_under: np.ndarray) -> np.ndarray:
    """Right-hand side (-f, -f_0) of Definition 9."""
    return -np.concatenate([f_under, f0_under])


def permutation(L: int) -> np.ndarray:
    """Row permutation P of Section 3.5 (Eq. of the splitting D^jump + R^jump).

    P M lists first the rows whose identity block acts on the down-going
    unknowns (j = n and j = n+1 of layers 1..L-1, i.e. trace 2i and 2i+1 of
    interface i) and then those acting on the up-going ones (j = 0 and j = 1 of
    layers 2..L), so that row r of P M has its identity on unknown r.
    Returns perm with (P y)[r] = y[perm[r]] at trace granularity.
    """
    T = 2 * (L - 1)
    perm = np.empty(2 * T, dtype=np.int64)
    for i in range(L - 1):
        perm[2 * i] = 2 * i  # jump 2 of layer i   (identity on u_down trace 2i)
        perm[2 * i + 1] = T + 2 * i  # jump 4 of layer i   (identity on u_down trace 2i+1)
        perm[T + 2 * i] = T + 2 * i + 1  # jump 3 of layer i+1 (identity on u_up trace 2i)
        perm[T + 2 * i + 1] = 2 * i + 1  # jump 1 of layer i+1 (identity on u_up trace 2i+1)
    return perm


def apply_P(y: np.ndarray, L: int, nt: int) -> np.ndarray:
    perm = permutation(L)
    return y.reshape(-1, nt)[perm].reshape(-1)


class Splitting:
    """P M = D + R (Section 3.5): D keeps the down-down and up-up couplings, R the rest."""

    def __init__(self, system: BlockSystem, L: int):
        self.S, self.L, self.nt = system, L, system.nt
        self.T = 2 * (L - 1)
        self.perm = permutation(L)
        # permuted system: row r of P M is row perm[r] of M
        self.PM = BlockSystem(system.nrows, system.ncols, system.nt)
        for r in range(system.nrows):
            self.PM.add(r, system.rows[self.perm[r]])

    def _side(self, idx: int) -> int:
        return 0 if idx < self.T else 1

    def in_D(self, r: int, c: int) -> bool:
        return self._side(r) == self._side(c)

    def in_R(self, r: int, c: int) -> bool:
        return self._side(r) != self._side(c)

    def apply_D(self, x):
        return self.PM.apply(x, self.in_D)

    def apply_R(self, x):
        return self.PM.apply(x, self.in_R)

    def solve_D(self, b: np.ndarray) -> np.ndarray:
        """D^{-1} b by block back-substitution (Section 4.1).

        D_down is block lower triangular and D_up block upper triangular,
        both with -I on the diagonal; each half is solved in its own order
        (top-down sweep for the down-going traces, bottom-up for the up-going).
        """
        nt, T = self.nt, self.T
        B = b.reshape(-1, nt)
        X = np.zeros_like(B)
        order = list(range(T)) + list(range(2 * T - 1, T - 1, -1))
        done = set()
        for r in order:
            acc = B[r].copy()
            diag_seen = False
            for c, blk in self.PM.rows[r]:
                if not self.in_D(r, c):
                    continue
                if c == r:
                    assert np.isscalar(blk) and blk == -1, "diagonal of D must be -I"
                    diag_seen = True
                    continue
                assert c in done, "D is not triangular in the sweep order"
                acc -= blk @ X[c]
            assert diag_seen
            X[r] = -acc
            done.add(r)
        return X.reshape(-1)


def gauss_seidel_preconditioner(split: Splitting, ftilde: np.ndarray, n_it: int = 2) -> np.ndarray:
    """Algorithm 4: u^0 = 0; u^{k+1} = D^{-1}(P f~ - R u^k), n_it times."""
    Pf = apply_P(ftilde, split.L, split.nt)
    u = np.zeros_like(Pf)
    for _ in range(n_it):
        u = split.solve_D(Pf - split.apply_R(u))
    return u


def gauss_seidel_iteration(split: Splitting, ftilde: np.ndarray, tol: float, max_it: int = 1000):
    """Algorithm 3: the same update, repeated while ||u^{k+1} - u^k|| / ||u^k|| > tol.

    Returns (u, iterations)."""
    Pf = apply_P(ftilde, split.L, split.nt)
    u = np.zeros_like(Pf)
    for k in range(1, max_it + 1):
        u_new = split.solve_D(Pf - split.apply_R(u))
        nrm = np.linalg.norm(u)
        change = np.linalg.norm(u_new - u) / nrm if nrm > 0 else np.inf
        u = u_new
        if change <= tol:
            return u, k
    return u, max_it


def collapse(u_pol: np.ndarray, L: int, nt: int) -> np.ndarray:
    """u = u_up + u_down (Section 3.2)."""
    T = 2 * (L - 1)
    U = u_pol.reshape(2 * T, nt)
    return (U[:T] + U[T:]).reshape(-1)


def extrapolator_up(G_next: dict) -> np.ndarray:
    """E_up_{l,l+1} = G^{l+1}(z_1, z_1)^{-1} G^{l+1}(z_1, z_0) (Definition 6)."""
    return np.linalg.solve(G_next[(1, 1)], G_next[(1, 0)])


def extrapolator_down(G: dict, n: int) -> np.ndarray:
    """E_down_{l,l+1} = G^l(z_n, z_n)^{-1} G^l(z_n, z_{n+1}) (Definition 6)."""
    return np.linalg.solve(G[(n, n)], G[(n, n + 1)])
