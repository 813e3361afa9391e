"""Section 2.3: interface Green's matrices, incomplete Green's integrals, Newton potential.

Test infrastructure: see the package docstring.

Definition 1 with the discrete delta of value 1/h^2 gives, for target row j
and source row k of layer l,

    G^l(z_j, z_k) = (1/h) [ (H^l)^{-1} ]_{(., j), (., k)}        (n_t x n_t),

the factor h of the quadrature in Definition 1 times the 1/h^2 of the delta.
Blocks are extracted by solving the local problem with columns of the
identity placed on row k (Algorithm 1, "extract Green's functions").
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from .discretization import Layer, Problem, local_operator


class LocalSolver:
    """Sparse LU of H^l (Algorithm 1, "factorize local problems")."""

    def __init__(self, prob: Problem, layer: Layer):
        self.prob = prob
        self.layer = layer
        self.H = local_operator(prob, layer)
        self.lu = spla.splu(self.H.tocsc())

    def solve(self, rhs: np.ndarray) -> np.ndarray:
        """(H^l)^{-1} rhs for rhs of shape (nloc, n_t) or (nloc*n_t, k)."""
        nt = self.prob.nt
        if rhs.ndim == 2 and rhs.shape == (self.layer.nloc, nt):
            return self.lu.solve(rhs.reshape(-1).astype(np.complex128)).reshape(self.layer.nloc, nt)
        return self.lu.solve(np.asarray(rhs, dtype=np.complex128))


def trace_rows(layer: Layer, L: int) -> list[int]:
    """Paper row indices j of the traces that layer l owns: {0, 1} if it has a
    top interface, {n, n+1} if it has a bottom interface (Definition 4)."""
    rows = []
    if layer.index > 0:
        rows += [0, 1]
    if layer.index < L - 1:
        rows += [layer.n, layer.n + 1]
    return rows


def green_blocks(solver: LocalSolver, L: int, sources=None, targets=None) -> dict:
    """G^l(z_j, z_k) for j, k in the layer's trace rows (Definition 1, Algorithm 1).

    Returns {(j, k): n_t x n_t array}.  ``sources``/``targets`` restrict the
    paper row indices used (default: the layer's trace rows).
    """
    layer, prob = solver.layer, solver.prob
    nt, h = prob.nt, prob.h
    sources = trace_rows(layer, L) if sources is None else list(sources)
    targets = trace_rows(layer, L) if targets is None else list(targets)
    out = {}
    for k in sources:
        rhs = np.zeros((layer.nloc * nt, nt), dtype=np.complex128)
        rk = layer.row(k)
        rhs[rk * nt + np.arange(nt), np.arange(nt)] = 1.0
        X = solver.solve(rhs)  # columns of (H^l)^{-1} at row k
        for j in targets:
            rj = layer.row(j)
            out[(j, k)] = X[rj * nt : (rj + 1) * nt, :] / h
    return out


def green_column(solver: LocalSolver, j_rows, k: int, col: int) -> dict:
    """One column (source node ``col`` on row k) of G^l(z_j, z_k) for each j in j_rows.

    Used to sample blocks at sizes where extracting all of them is too slow.
    """
    layer, prob = solver.layer, solver.prob
    nt, h = prob.nt, prob.h
    rhs = np.zeros(layer.nloc * nt, dtype=np.complex128)
    rhs[layer.row(k) * nt + col] = 1.0
    x = solver.solve(rhs[:, None])[:, 0]
    return {j: x[layer.row(j) * nt : (layer.row(j) + 1) * nt] / h for j in j_rows}


def incomplete_green_down(G: dict, j: int, v0: np.ndarray, v1: np.ndarray, h: float) -> np.ndarray:
    """Down-going incomplete Green's integral (Definition 2):

    G_down_j(v_0, v_1) = -G(z_j, z_0) (v_1 - v_0)/h + ((G(z_j, z_1) - G(z_j, z_0))/h) v_0.
    """
    return -G[(j, 0)] @ ((v1 - v0) / h) + ((G[(j, 1)] - G[(j, 0)]) / h) @ v0


def incomplete_green_up(G: dict, j: int, n: int, vn: np.ndarray, vn1: np.ndarray, h: float) -> np.ndarray:
    """Up-going incomplete Green's integral (Definition 2):

    G_up_j(v_n, v_{n+1}) = G(z_j, z_{n+1}) (v_{n+1} - v_n)/h - ((G(z_j, z_{n+1}) - G(z_j, z_n))/h) v_{n+1}.
    """
    return G[(j, n + 1)] @ ((vn1 - vn) / h) - ((G[(j, n + 1)] - G[(j, n)]) / h) @ vn1


def restrict_source(f: np.ndarray, layer: Layer) -> np.ndarray:
    """f^l = f chi_{Omega^l} on the local grid, zero in the padded PML (Algorithm 2)."""
    nt = f.shape[1]
    out = np.zeros((layer.nloc, nt), dtype=np.complex128)
    out[layer.pad_top : layer.pad_top + layer.n] = f[layer.start : layer.start + layer.n]
    return out


def newton_potential(solver: LocalSolver, f: np.ndarray) -> np.ndarray:
    """N^l f^l := (H^l)^{-1} f^l on the whole local grid (Algorithm 2, "solve local problems").

    Reading: Definition 3 writes the quadrature sum with the Green's matrices
    of Definition 1, which carries an extra factor h relative to its own claim
    H N f = f; Algorithm 2 defines the potential as the local solve, which is
    what is used here.
    """
    return solver.solve(restrict_source(f, solver.layer))


def grf_forcing(layer: Layer, nt: int, h: float, f: np.ndarray, traces: dict) -> np.ndarray:
    """Right-hand side of the PDE form of the discrete GRF (Section 2.3):

    H^l v = f^l + delta(z_1 - z) v_0 - delta(z_0 - z) v_1 - delta(z_{n+1} - z) v_n + delta(z_n - z) v_{n+1},

    delta = 1/h^2 on a row.  ``traces`` maps the paper row index (0, 1, n, n+1)
    to a trace; missing rows (no interface on that side) contribute nothing.
    """
    rhs = restrict_source(f, layer)
    n = layer.n
    inv_h2 = 1.0 / (h * h)
    if 0 in traces:
        rhs[layer.row(1)] += inv_h2 * traces[0]
        rhs[layer.row(0)] -= inv_h2 * traces[1]
    if n in traces:
        rhs[layer.row(n + 1)] -= inv_h2 * traces[n]
        rhs[layer.row(n)] += inv_h2 * traces[n + 1]
    return rhs


def reconstruct_layer(solver: LocalSolver, f: np.ndarray, traces: dict) -> np.ndarray:
    """Local field v^l from its interface traces (Algorithm 2, last loop).

    Evaluates the discrete GRF (Lemma 1) by the local sparse solve with the
    forcing of the PDE form, as Section 2.3 describes.  Returns the whole
    local grid (nloc, n_t); rows 1..n are the layer's part of the solution.
    """
    layer, prob = solver.layer, solver.prob
    return solver.solve(grf_forcing(layer, prob.nt, prob.h, f, traces))
