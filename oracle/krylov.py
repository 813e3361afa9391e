"""Section 4.2: GMRES with the Gauss-Seidel preconditioner.

Test infrastructure: see the package docstring.

The paper uses plain GMRES (Arnoldi with modified Gram-Schmidt, Givens
rotations on the Hessenberg matrix, no restart) and analyses the left
preconditioned operator.  Both the left preconditioned form and the right
preconditioned (flexible) form are written here; the two reach the same
solution of the linear system.  Start vector x_0 = 0.
"""
from __future__ import annotations

import numpy as np


def _givens(a: complex, b: complex):
    """Complex Givens rotation (c real, s complex) with [c s; -conj(s) c] (a; b) = (r; 0)."""
    if b == 0:
        return 1.0, 0.0 + 0.0j
    if a == 0:
        return 0.0, np.conj(b) / abs(b)
    t = np.hypot(abs(a), abs(b))
    c = abs(a) / t
    s = (a / abs(a)) * np.conj(b) / t
    return c, s


def _arnoldi_solve(apply_op, r0: np.ndarray, tol_abs: float, max_it: int, prec=None):
    """Arnoldi (MGS) + Givens least squares on span{r0, (op) r0, ...}.

    apply_op(v) returns the operator applied to v; when ``prec`` is given the
    Krylov vectors are preconditioned first (flexible form) and the returned
    correction is Z y, otherwise V y.  Stops as soon as the least-squares
    residual |g_{k+1}| <= tol_abs.  Returns (correction, iterations, history).
    """
    n = r0.shape[0]
    beta = np.linalg.norm(r0)
    hist = [beta]
    if beta <= tol_abs or max_it == 0:
        return np.zeros(n, dtype=np.complex128), 0, hist
    V = np.zeros((max_it + 1, n), dtype=np.complex128)
    Z = np.zeros((max_it, n), dtype=np.complex128) if prec is not None else None
    Hm = np.zeros((max_it + 1, max_it), dtype=np.complex128)
    cs = np.zeros(max_it)
    sn = np.zeros(max_it, dtype=np.complex128)
    g = np.zeros(max_it + 1, dtype=np.complex128)
    g[0] = beta
    V[0] = r0 / beta
    k = 0
    for k in range(max_it):
        if prec is not None:
            Z[k] = prec(V[k])
            w = apply_op(Z[k])
        else:
            w = apply_op(V[k])
        for i in range(k + 1):  # modified Gram-Schmidt
            Hm[i, k] = np.vdot(V[i], w)
            w = w - Hm[i, k] * V[i]
        Hm[k + 1, k] = np.linalg.norm(w)
        if Hm[k + 1, k] != 0:
            V[k + 1] = w / Hm[k + 1, k]
        for i in range(k):  # previous rotations on the new column
            t = cs[i] * Hm[i, k] + sn[i] * Hm[i + 1, k]
            Hm[i + 1, k] = -np.conj(sn[i]) * Hm[i, k] + cs[i] * Hm[i + 1, k]
            Hm[i, k] = t
        cs[k], sn[k] = _givens(Hm[k, k], Hm[k + 1, k])
        Hm[k, k] = cs[k] * Hm[k, k] + sn[k] * Hm[k + 1, k]
        Hm[k + 1, k] = 0.0
        g[k + 1] = -np.conj(sn[k]) * g[k]
        g[k] = cs[k] * g[k]
        hist.append(abs(g[k + 1]))
        if abs(g[k + 1]) <= tol_abs:
            break
    m = k + 1
    y = np.zeros(m, dtype=np.complex128)
    for i in range(m - 1, -1, -1):  # back substitution on the triangular R
        y[i] = (g[i] - Hm[i, i + 1 : m] @ y[i + 1 : m]) / Hm[i, i]
    basis = Z if prec is not None else V
    return y @ basis[:m], m, hist


def gmres_left(A, b: np.ndarray, Minv, tol: float, max_it: int):
    """GMRES on M^{-1} A x = M^{-1} b (left preconditioned, Section 4.2).

    Stops when ||M^{-1}(b - A x)|| <= tol ||M^{-1} b||.  Returns (x, its, history)."""
    r0 = Minv(b)
    dx, its, hist = _arnoldi_solve(lambda v: Minv(A(v)), r0, tol * np.linalg.norm(r0), max_it)
    return dx, its, hist


def fgmres_right(A, b: np.ndarray, Minv, tol: float, max_it: int, max_cycles: int = 5):
    """Flexible GMRES with right preconditioning: A M^{-1} y = b, x = M^{-1} y.

    Stops when the least-squares estimate is <= tol ||b||, then confirms with
    the explicit residual ||b - A x|| / ||b||; when rounding makes the two
    disagree the cycle restarts from the current x.  Returns
    (x, total iterations, true relative residual, history)."""
    x = np.zeros_like(b)
    bnorm = np.linalg.norm(b)
    total, hist = 0, []
    for _ in range(max_cycles):
        r = b - A(x) if total else b.copy()
        rel = np.linalg.norm(r) / bnorm
        if rel <= tol or total >= max_it:
            return x, total, rel, hist
        dx, its, h = _arnoldi_solve(A, r, tol * bnorm, max_it - total, prec=Minv)
        x = x + dx
        total += its
        hist += h
    r = b - A(x)
    return x, total, np.linalg.norm(r) / bnorm, hist
