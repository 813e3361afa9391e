"""Uneven batch: independent problems solved concurrently (pt_solve_many).

Each instance has its own medium, grid, layer count and sources; solving
them together must give exactly what solving each alone gives (the same
kernels on the same data, only overlapped in time: the concurrent contexts
take the per-step preconditioner sweeps, so the single solves are asked for
them too), and each must match the oracle's global direct solve within the
mixed tolerance.
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import discretization as D
from oracle import solver as S

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_uneven_batch_equals_single_solves_and_oracle():
    from paper_1410_5910_gb300 import PT_MIXED_FP32, PT_OPT_SWEEP, PolarTrace, solve_many

    cases = W.uneven_batch(count=4, seed=7, nmin=21, nmax=41, Lmin=3, Lmax=5, npml=8, smax=3)
    solvers, fs, refs = [], [], []
    for wl in cases:
        c = wl.c_ext()
        om = wl.omega(c)
        prob = D.make_problem(c, wl.npml, wl.h, om)
        sv = PolarTrace(wl.nx, wl.nz, wl.npml, wl.L, wl.h, om, torch.from_numpy(c).cuda(), pml_C=prob.C,
                        precision=PT_MIXED_FP32, max_sources=len(wl.sources), stream=torch.cuda.Stream())
        f = wl.f()
        solvers.append(sv)
        fs.append(torch.from_numpy(f).cuda())
        refs.append(S.global_solve(prob, f))
    assert len({(wl.nx, wl.L, len(wl.sources)) for wl in cases}) > 1  # really uneven
    us, its, rels = solve_many(solvers, fs, tol=1e-9)
    for k, (sv, f, wl) in enumerate(zip(solvers, fs, cases)):
        sv.set_option(PT_OPT_SWEEP, 1)
        u1, _, it1, rel1 = sv.solve(f, tol=1e-9)
        torch.cuda.synchronize()
        assert torch.equal(us[k], u1) and its[k] == it1
        for s in range(f.shape[0]):
            assert rels[k][s] <= 1e-9
            assert _rel(us[k][s].cpu().numpy(), refs[k][s]) < 1e-5
