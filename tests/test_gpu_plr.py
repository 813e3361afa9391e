"""GPU partitioned low-rank blocks (Section 5.1) against the oracle.

The library compresses each interface block with Algorithm 5 using a
randomized SVD (as Section 7 does); the oracle uses the exact SVD.  The two
trees may differ where a singular value sits at the threshold, so the checks
are on what both must satisfy: the compressed operators reproduce the dense
ones to within the truncation (eps times the number of leaves), the storage
is close to the oracle's, and the solve reaches the oracle's volume field.
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import discretization as D
from oracle import plr
from oracle import solver as S

pytestmark = pytest.mark.gpu


def _rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _mk(wl, precision=0, rmax=6, eps=1e-9):
    from paper_1410_5910_gb300 import PolarTrace

    c = wl.c_ext()
    om = wl.omega(c)
    prob = D.make_problem(c, wl.npml, wl.h, om)
    solver = PolarTrace(wl.nx, wl.nz, wl.npml, wl.L, wl.h, om, torch.from_numpy(c).cuda(), pml_C=prob.C,
                        precision=precision, plr=True, plr_eps=eps, plr_rmax=rmax)
    return prob, solver


CASE = W.small_case(60, 70, 8, 3, medium="grf", seed=31)


@pytest.fixture(scope="module")
def fp64():
    prob, solver = _mk(CASE)
    off = S.precompute(prob, CASE.L)
    return prob, solver, off


def test_compressed_operators_reproduce_dense_ones(fp64):
    prob, solver, off = fp64
    g = np.random.default_rng(3)
    x = g.standard_normal((1, solver.T4, solver.nt)) + 1j * g.standard_normal((1, solver.T4, solver.nt))
    xt = torch.from_numpy(x).cuda()
    sp_ = off.split
    for which, ref in (("matvec", sp_.PM.apply(x[0].ravel())), ("R", sp_.apply_R(x[0].ravel())),
                       ("Dinv", sp_.solve_D(x[0].ravel()))):
        got = solver.apply(which, xt, working=True).cpu().numpy()[0].ravel()
        assert _rel(got, ref) < 1e-7, which
        dense = solver.apply(which, xt, working=False).cpu().numpy()[0].ravel()
        assert _rel(dense, ref) < 1e-11, which


def test_compression_matches_oracle_storage(fp64):
    prob, solver, off = fp64
    stored, leaves = solver.plr_stats()
    assert leaves > len(off.blocks) * 4  # the trees do split
    oracle_stored = 0
    for G in off.blocks:
        for blk in G.values():
            oracle_stored += plr.compressed_entries(plr.compress(blk / prob.h, 6, 1e-9))
    assert 0.75 * oracle_stored <= stored <= 1.25 * oracle_stored, (stored, oracle_stored)
    dense = sum(blk.size for G in off.blocks for blk in G.values())
    assert stored < dense


@pytest.mark.parametrize("precision,tol_field", [(0, 1e-6), (1, 1e-5)])
def test_solve_with_compressed_blocks(fp64, precision, tol_field):
    prob, _, off = fp64
    _, solver = _mk(CASE, precision=precision)
    f = CASE.f()
    u, tr, its, rel = solver.solve(torch.from_numpy(f).cuda(), tol=1e-9)
    u_ref = S.global_solve(prob, f[0])
    mask = D.physical_mask(prob, CASE.nx, CASE.nz)
    assert rel[0] <= 1e-9  # explicit residual with the dense FP64 operator
    assert _rel(u.cpu().numpy()[0][mask], u_ref[mask]) < tol_field
