"""Algorithms 1 and 2 with the polarized jump system: the oracle's end-to-end solve.

Test infrastructure: see the package docstring.

Also the plain definition of what the method computes: the global sparse
direct solve of H u = f (Theorem 1 and Proposition 1 say the method reaches
exactly this discrete solution).
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.sparse.linalg as spla

from . import green, integral, krylov, polarized
from .discretization import Problem, check_partition, global_operator, layer_partition, make_layer


def global_solve(prob: Problem, f: np.ndarray) -> np.ndarray:
    """u = H^{-1} f on the extended grid (Section 2.1), f of shape (N_z, n_t) or (S, N_z, n_t)."""
    lu = spla.splu(global_operator(prob).tocsc())
    if f.ndim == 2:
        return lu.solve(f.reshape(-1).astype(np.complex128)).reshape(f.shape)
    F = f.reshape(f.shape[0], -1).T.astype(np.complex128)
    return lu.solve(F).T.reshape(f.shape)


def global_traces(u: np.ndarray, nc: np.ndarray) -> np.ndarray:
    """Restriction of a volume field to the interfaces: trace 2i = row n of layer i,
    trace 2i+1 = row n+1 of layer i (ordering of Definition 4)."""
    out = []
    for i in range(1, len(nc) - 1):
        s = int(nc[i])
        out += [u[s - 1], u[s]]
    return np.concatenate(out)


@dataclasses.dataclass
class Offline:
    """Algorithm 1: local factorizations, interface Green's matrices, systems."""

    prob: Problem
    nc: np.ndarray
    layers: list
    solvers: list
    blocks: list
    ns: list
    system: integral.BlockSystem
    split: polarized.Splitting

    @property
    def L(self) -> int:
        return len(self.layers)


def precompute(prob: Problem, L: int, nc: np.ndarray | None = None) -> Offline:
    """Algorithm 1 (offline): partition, local LU, Green's extraction, form the system."""
    nc = layer_partition(prob.Nz, L) if nc is None else np.asarray(nc)
    check_partition(prob.Nz, prob.npml, nc)
    layers = [make_layer(prob, nc, l) for l in range(L)]
    solvers = [green.LocalSolver(prob, lay) for lay in layers]
    blocks = [green.green_blocks(s, L) for s in solvers]
    ns = [lay.n for lay in layers]
    system = polarized.polarized_jump_system(blocks, ns, prob.h, prob.nt)
    return Offline(prob, nc, layers, solvers, blocks, ns, system, polarized.Splitting(system, L))


def newton_traces(off: Offline, f: np.ndarray):
    """Local solves N^l f^l and their values at the trace rows (Algorithm 2)."""
    out = []
    for lay, s in zip(off.layers, off.solvers):
        fl = green.restrict_source(f, lay)
        if not np.any(fl):
            vol = np.zeros((lay.nloc, off.prob.nt), dtype=np.complex128)
        else:
            vol = s.solve(fl)
        out.append({j: vol[lay.row(j)] for j in green.trace_rows(lay, off.L)})
    return out


def polarized_rhs(off: Offline, f: np.ndarray) -> np.ndarray:
    """(-f, -f_0) of Definition 9 from the local Newton potentials."""
    nt = off.prob.nt
    nw = newton_traces(off, f)
    fu = integral.integral_rhs(nw, off.ns, nt)
    f0 = integral.integral_rhs(nw, off.ns, nt, outside=True)
    return polarized.polarized_rhs(fu, f0)


def reconstruct(off: Offline, f: np.ndarray, traces: np.ndarray) -> np.ndarray:
    """Volume field from the (collapsed) traces, concatenated over layers (Algorithm 2)."""
    prob, nt = off.prob, off.prob.nt
    U = traces.reshape(-1, nt)
    u = np.zeros((prob.Nz, nt), dtype=np.complex128)
    for l, (lay, s) in enumerate(zip(off.layers, off.solvers)):
        tr = {}
        if l > 0:
            tr[0], tr[1] = U[2 * (l - 1)], U[2 * (l - 1) + 1]
        if l < off.L - 1:
            tr[lay.n], tr[lay.n + 1] = U[2 * l], U[2 * l + 1]
        v = green.reconstruct_layer(s, f, tr)
        u[lay.start : lay.start + lay.n] = v[lay.pad_top : lay.pad_top + lay.n]
    return u


@dataclasses.dataclass
class SolveResult:
    u: np.ndarray  # volume field (N_z, n_t)
    traces_pol: np.ndarray  # (u_down, u_up)
    iterations: int
    true_relres: float
    history: list


def online_solve(off: Offline, f: np.ndarray, tol: float = 1e-7, max_it: int = 60, n_it: int = 2,
                 form: str = "right") -> SolveResult:
    """Algorithm 2 with the polarized jump system solved by preconditioned GMRES (Section 4.2)."""
    b = polarized_rhs(off, f)
    A = off.system.apply
    Minv = lambda v: polarized.gauss_seidel_preconditioner(off.split, v, n_it)  # noqa: E731
    if form == "right":
        x, its, rel, hist = krylov.fgmres_right(A, b, Minv, tol, max_it)
    else:
        x, its, hist = krylov.gmres_left(A, b, Minv, tol, max_it)
        rel = np.linalg.norm(b - A(x)) / np.linalg.norm(b)
    u = reconstruct(off, f, polarized.collapse(x, off.L, off.prob.nt))
    return SolveResult(u, x, its, rel, hist)


def global_factor(prob: Problem):
    """Sparse LU of the global H (the factorization inside ``global_solve``), for timing
    the per-source back-substitution separately from the factorization."""
    return spla.splu(global_operator(prob).tocsc())
