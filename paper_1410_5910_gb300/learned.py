"""Training data for the learned preconditioner correction, produced by the solver.

For sources f the converged traces x* and the iterates x_k after k GMRES
iterations give errors e_k = x* - x_k and residuals r_k = P b - P M x_k =
P M e_k (Section 4.2).  Every step runs in the library (solves and the exact
FP64 matvec); this module only strings the calls together.
"""
from __future__ import annotations

import torch


def solver_pairs(solver, f: torch.Tensor, iters=(0, 1, 2, 3, 4), tol: float = 1e-12):
    """(r, e) pairs, each (len(iters) * S, 4(L-1), n_t) complex128 on the device."""
    _, xs, _, _ = solver.solve(f, tol=tol, want_u=False)
    rs, es = [], []
    for k in iters:
        if k == 0:
            e = xs.clone()
        else:
            _, xk, _, _ = solver.solve(f, tol=1e-15, max_it=k, want_u=False, allow_not_converged=True)
            e = xs - xk
        rs.append(solver.matvec(e.contiguous()))
        es.append(e)
    return torch.cat(rs).contiguous(), torch.cat(es).contiguous()


def gate(solver, f_val: torch.Tensor, tol: float = 1e-7):
    """Keep the learned correction only where it pays: solve the validation sources
    with and without it (the FP64 true residual judges both) and leave
    PT_OPT_LEARNED on only if the corrected solves took fewer GMRES iterations in
    total.  Returns (iterations plain, iterations corrected, kept)."""
    from . import PT_OPT_LEARNED

    solver.set_option(PT_OPT_LEARNED, 0)
    _, _, its0, _ = solver.solve(f_val, tol=tol, want_u=False)
    solver.set_option(PT_OPT_LEARNED, 1)
    _, _, its1, _ = solver.solve(f_val, tol=tol, want_u=False, allow_not_converged=True)
    keep = sum(its1) < sum(its0)
    solver.set_option(PT_OPT_LEARNED, 1 if keep else 0)
    return its0, its1, keep
