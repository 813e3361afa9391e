"""Batched sources on the tensor cores (PT_MIXED_TC) against the oracle.

The block products run as FP16 x FP16 -> FP32 tensor-core contractions with
power-of-two scales: one pass (~11-bit operands) in the preconditioner, the
three-pass hi/lo split (~22-bit operands, FP32 accumulation) in the GMRES
matvec.  Tolerances follow from those precisions; the solve must meet the
1e-5 volume-error bound of the mixed forms.  The FP64 volume residual
||f - H u|| / ||f|| is pinned on the oracle's exact solution.
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import discretization as D
from oracle import solver as S

pytestmark = pytest.mark.gpu

CASE = W.small_case(40, 60, 8, 3, medium="grf", seed=11)


def _rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def setup():
    from paper_1410_5910_gb300 import PT_MIXED_TC, PolarTrace

    c = CASE.c_ext()
    om = CASE.omega(c)
    prob = D.make_problem(c, CASE.npml, CASE.h, om)
    solver = PolarTrace(CASE.nx, CASE.nz, CASE.npml, CASE.L, CASE.h, om, torch.from_numpy(c).cuda(), pml_C=prob.C,
                        precision=PT_MIXED_TC, max_sources=160, max_krylov=40)
    off = S.precompute(prob, CASE.L)
    return prob, solver, off


@pytest.mark.parametrize("nsrc", [8, 64, 150])
def test_tensor_core_operators(setup, nsrc):
    prob, solver, off = setup
    g = np.random.default_rng(nsrc)
    x = g.standard_normal((nsrc, solver.T4, solver.nt)) + 1j * g.standard_normal((nsrc, solver.T4, solver.nt))
    xt = torch.from_numpy(x).cuda()
    sp_ = off.split
    got_R = solver.apply("R", xt, working=True).cpu().numpy()
    got_M = solver.apply("matvec", xt, working=True).cpu().numpy()
    got_D = solver.apply("Dinv", xt, working=True).cpu().numpy()
    for s in (0, nsrc // 2, nsrc - 1):
        xs = x[s].ravel()
        assert _rel(got_R[s].ravel(), sp_.apply_R(xs)) < 5e-3          # one FP16 pass
        assert _rel(got_M[s].ravel(), sp_.PM.apply(xs)) < 2e-5         # three-pass split
        assert _rel(got_D[s].ravel(), sp_.solve_D(xs)) < 2e-2          # sweeps of one-pass products


def test_volume_residual_of_exact_solution_is_roundoff(setup):
    prob, solver, off = setup
    f = CASE.f()
    u = S.global_solve(prob, f[0])
    rel = solver.volume_residual(torch.from_numpy(f).cuda(), torch.from_numpy(u[None]).cuda())
    assert rel[0] < 1e-12
    # and it sees a perturbation of size eps
    up = u.copy()
    up[10, 10] += 1e-3 * np.abs(u).max()
    rel = solver.volume_residual(torch.from_numpy(f).cuda(), torch.from_numpy(up[None]).cuda())
    assert rel[0] > 1e-6


def test_batched_tensor_core_solve_meets_mixed_tolerance(setup):
    prob, solver, off = setup
    g = np.random.default_rng(5)
    pos = [(int(g.integers(1, CASE.nx + 1)), int(g.integers(1, CASE.nz + 1))) for _ in range(24)]
    f = W.point_sources(CASE.nt, CASE.Nz, CASE.npml, CASE.h, pos)
    ft = torch.from_numpy(f).cuda()
    u, tr, its, rel = solver.solve(ft, tol=1e-7)
    ref = S.global_solve(prob, f)
    mask = D.physical_mask(prob, CASE.nx, CASE.nz)
    un = u.cpu().numpy()
    for s in range(len(pos)):
        assert rel[s] <= 1e-7
        assert _rel(un[s][mask], ref[s][mask]) < 1e-5
    vres = solver.volume_residual(ft, u)
    assert max(vres) < 1e-5
