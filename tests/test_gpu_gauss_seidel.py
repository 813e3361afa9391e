"""Gauss-Seidel on the GPU: Algorithm 3 as a solver and Algorithm 4 with other n_it.

Both run the sweeps D^{-1} and the coupling R of Section 4.1 (FP64 blocks), so
they are compared with the oracle's restatements of the same algorithms
(oracle.polarized.gauss_seidel_iteration / gauss_seidel_preconditioner) at
FP64 rounding level, and the solutions with the global direct solve.
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import discretization as D
from oracle import polarized
from oracle import solver as S

pytestmark = pytest.mark.gpu


def _rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _mk(wl, gs_iters=2, precision=0, max_sources=1):
    from paper_1410_5910_gb300 import PolarTrace

    c = wl.c_ext()
    om = wl.omega(c)
    prob = D.make_problem(c, wl.npml, wl.h, om)
    solver = PolarTrace(wl.nx, wl.nz, wl.npml, wl.L, wl.h, om, torch.from_numpy(c).cuda(), pml_C=prob.C,
                        precision=precision, max_sources=max_sources, gs_iters=gs_iters)
    return prob, solver


CASES = [
    W.small_case(40, 60, 8, 3, medium="grf", seed=11),
    W.small_case(37, 45, 6, 4, medium="constant", sources=((5, 30),)),
]


@pytest.fixture(scope="module", params=range(len(CASES)))
def case(request):
    wl = CASES[request.param]
    c = wl.c_ext()
    prob = D.make_problem(c, wl.npml, wl.h, wl.omega(c))
    off = S.precompute(prob, wl.L)
    return wl, prob, off


@pytest.mark.parametrize("n_it", [1, 3])
def test_preconditioner_with_other_n_it_matches_oracle(case, n_it):
    wl, prob, off = case
    _, solver = _mk(wl, gs_iters=n_it)
    sp_ = off.split
    g = np.random.default_rng(3 + n_it)
    x = g.standard_normal((1, solver.T4, solver.nt)) + 1j * g.standard_normal((1, solver.T4, solver.nt))
    unperm = np.empty_like(x[0])
    unperm[sp_.perm] = x[0]  # the oracle's Algorithm 4 takes the unpermuted residual
    ref = polarized.gauss_seidel_preconditioner(sp_, unperm.ravel(), n_it)
    got = solver.precond(torch.from_numpy(x).cuda()).cpu().numpy()[0].ravel()
    assert _rel(got, ref) < 1e-11


@pytest.mark.parametrize("n_it", [1, 3])
def test_gmres_with_other_n_it_reaches_the_global_solve(case, n_it):
    wl, prob, off = case
    _, solver = _mk(wl, gs_iters=n_it)
    f = wl.f()
    u_ref = S.global_solve(prob, f[0])
    u, _, its, rel = solver.solve(torch.from_numpy(f).cuda(), tol=1e-10)
    assert rel[0] <= 1e-10
    assert _rel(u.cpu().numpy()[0], u_ref) < 1e-6
    ores = S.online_solve(off, f[0], tol=1e-10, n_it=n_it)
    assert abs(ores.iterations - its[0]) <= 1


def test_gauss_seidel_solver_matches_oracle_iteration(case):
    wl, prob, off = case
    _, solver = _mk(wl)
    f = wl.f()
    tol = 1e-11
    ref_u, ref_its = polarized.gauss_seidel_iteration(off.split, S.polarized_rhs(off, f[0]), tol, max_it=400)
    u, tr, its, rel = solver.solve_gs(torch.from_numpy(f).cuda(), tol=tol, max_it=400)
    # the same iteration in the same order: the same count (+-1 where the change sits at the threshold)
    assert abs(its[0] - ref_its) <= 1
    assert _rel(tr.cpu().numpy()[0].ravel(), ref_u) < 1e-9
    # and the solution of the discrete problem (Theorem 1): the global direct solve
    u_glob = S.global_solve(prob, f[0])
    assert rel[0] < 1e-9
    assert _rel(u.cpu().numpy()[0], u_glob) < 1e-7


def test_gauss_seidel_zero_source_and_batch(case):
    wl, prob, off = case
    _, solver = _mk(wl, max_sources=3)
    f = np.concatenate([np.zeros((1, wl.Nz, wl.nt), np.complex128),
                        W.point_sources(wl.nt, wl.Nz, wl.npml, wl.h, [(3, 4), (wl.nx - 2, wl.nz - 1)])])
    u, _, its, rel = solver.solve_gs(torch.from_numpy(f).cuda(), tol=1e-10, max_it=400)
    un = u.cpu().numpy()
    assert np.all(un[0] == 0) and its[0] == 1
    u_glob = S.global_solve(prob, f[1:])
    for s in (1, 2):
        assert _rel(un[s], u_glob[s - 1]) < 1e-6


def test_gauss_seidel_reports_non_convergence(case):
    from paper_1410_5910_gb300 import PolarTraceError

    wl, prob, off = case
    _, solver = _mk(wl)
    f = torch.from_numpy(wl.f()).cuda()
    with pytest.raises(PolarTraceError):
        solver.solve_gs(f, tol=1e-14, max_it=2)
    u, _, its, _ = solver.solve_gs(f, tol=1e-14, max_it=2, allow_not_converged=True)
    assert its[0] == 2 and torch.isfinite(torch.view_as_real(u)).all()
