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


# ---- source-batched FP32 local solves (right-hand side and reconstruction) ----
# The Schur inverses of the FP64 block factorization are rounded to complex64
# and the chains run in FP32: the right-hand side and the volume field carry
# FP32 rounding accumulated over 2 n_t steps (about 1e-6 on these grids, the
# same order as a direct FP32 emulation of the substitution), inside the 1e-5
# bound of the mixed forms.  Group widths 8, 16 and 32 are forced so that every
# kernel variant runs, with source counts that leave a ragged last group.

from oracle import polarized  # noqa: E402


def _mixed_sources(case, count, seed):
    g = np.random.default_rng(seed)
    pos = [(int(g.integers(1, case.nx + 1)), int(g.integers(1, case.nz + 1))) for _ in range(count - 1)]
    f = W.point_sources(case.nt, case.Nz, case.npml, case.h, pos)
    dense = W.random_sources(case.nt, case.Nz, case.npml, case.nx, case.nz, seed + 1, 1)  # excites every layer
    return np.concatenate([f, dense], axis=0)


@pytest.mark.parametrize("gw,count", [(8, 37), (16, 21), (32, 45)])
def test_batched_local_solves_match_oracle(setup, gw, count):
    from paper_1410_5910_gb300 import PT_OPT_LAYER_GROUP

    prob, solver, off = setup
    solver.set_option(PT_OPT_LAYER_GROUP, gw)
    try:
        f = _mixed_sources(CASE, count, 100 + gw)
        ft = torch.from_numpy(f).cuda()
        got = solver.rhs(ft).cpu().numpy()
        for s in (0, count // 2, count - 1):
            ref = polarized.apply_P(S.polarized_rhs(off, f[s]), off.L, prob.nt)
            assert _rel(got[s].ravel(), ref) < 1e-5
        u, tr, its, rel = solver.solve(ft, tol=1e-7)
        mask = D.physical_mask(prob, CASE.nx, CASE.nz)
        un = u.cpu().numpy()
        for s in (0, count // 2, count - 1):
            ref = S.global_solve(prob, f[s])
            assert rel[s] <= 1e-7
            assert _rel(un[s][mask], ref[mask]) < 1e-5
    finally:
        solver.set_option(PT_OPT_LAYER_GROUP, 0)


# a middle layer of 75 rows + 2 x 20 padded rows = 115 local rows: Sinv no longer
# fits twice in shared memory for 32 sources per CTA (single-buffered path)
TALL = W.small_case(30, 185, 20, 3, medium="grf", seed=12)


@pytest.mark.parametrize("gw", [8, 32])
def test_batched_local_solves_tall_layers(gw):
    from paper_1410_5910_gb300 import PT_MIXED_TC, PT_OPT_LAYER_GROUP, PolarTrace

    c = TALL.c_ext()
    om = TALL.omega(c)
    prob = D.make_problem(c, TALL.npml, TALL.h, om)
    solver = PolarTrace(TALL.nx, TALL.nz, TALL.npml, TALL.L, TALL.h, om, torch.from_numpy(c).cuda(), pml_C=prob.C,
                        precision=PT_MIXED_TC, max_sources=40, max_krylov=40)
    solver.set_option(PT_OPT_LAYER_GROUP, gw)
    f = _mixed_sources(TALL, 33, 7)
    u, tr, its, rel = solver.solve(torch.from_numpy(f).cuda(), tol=1e-7)
    mask = D.physical_mask(prob, TALL.nx, TALL.nz)
    un = u.cpu().numpy()
    for s in (0, 32):
        ref = S.global_solve(prob, f[s])
        assert rel[s] <= 1e-7
        assert _rel(un[s][mask], ref[mask]) < 1e-5
