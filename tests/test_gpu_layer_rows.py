"""A caller-chosen layer split (pt_params.layer_rows, Section 2.2: any increasing sequence of
interfaces) against the oracle run on the same split.

The split below is deliberately uneven (layers of 9 to 33 rows); the Green's blocks, the
right-hand side and the solves must match the oracle's, built with the same interface rows,
to the tolerances of the default split (FP64 1e-10 / 1e-6, mixed 1e-5 on the field).
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
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


WL = W.small_case(40, 60, 8, 4, medium="grf", seed=13, sources=((20, 40), (7, 2)))
ROWS = [33, 9, 20, 14]  # N_z = 60 + 16 = 76


@pytest.fixture(scope="module")
def uneven():
    assert sum(ROWS) == WL.Nz
    c = WL.c_ext()
    prob = D.make_problem(c, WL.npml, WL.h, WL.omega(c))
    nc = np.concatenate([[0], np.cumsum(ROWS)])
    off = S.precompute(prob, WL.L, nc=nc)
    return c, prob, off


def _solver(c, prob, precision):
    from paper_1410_5910_gb300 import PolarTrace

    return PolarTrace(WL.nx, WL.nz, WL.npml, WL.L, WL.h, WL.omega(c), torch.from_numpy(c).cuda(), pml_C=prob.C,
                      precision=precision, max_sources=2, layer_rows=ROWS)


def test_partition_follows_layer_rows():
    from paper_1410_5910_gb300 import layer_partition

    assert layer_partition(WL.nx, WL.nz, WL.npml, WL.L, layer_rows=ROWS) == [0, 33, 42, 62, 76]


def test_blocks_and_rhs_on_an_uneven_split(uneven):
    c, prob, off = uneven
    sv = _solver(c, prob, 0)
    for l, G in enumerate(off.blocks):
        for (j, k), blk in G.items():
            assert _rel(sv.block(l, j, k).cpu().numpy(), blk / prob.h) < 1e-10, (l, j, k)
    f = WL.f()
    got = sv.rhs(torch.from_numpy(f).cuda()).cpu().numpy()
    for s in range(2):
        ref = polarized.apply_P(S.polarized_rhs(off, f[s]), off.L, prob.nt)
        assert _rel(got[s].ravel(), ref) < 1e-11


@pytest.mark.parametrize("precision,tol,bound", [(0, 1e-10, 1e-6), (1, 1e-9, 1e-5), (2, 1e-7, 1e-5)])
def test_solves_on_an_uneven_split_reach_the_global_solve(uneven, precision, tol, bound):
    c, prob, off = uneven
    sv = _solver(c, prob, precision)
    f = WL.f()
    u, _, its, rel = sv.solve(torch.from_numpy(f).cuda(), tol=tol)
    ref = S.global_solve(prob, f)
    un = u.cpu().numpy()
    for s in range(2):
        assert rel[s] <= tol
        assert _rel(un[s], ref[s]) < bound
