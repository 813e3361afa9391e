"""The explicit restart residual of the tensor-core form by split products (PT_OPT_RESTART = 1).

Blocks and inputs are cut into five 7-bit integer slices (FP16-exact), the 15
slice pairs of weight >= 2^-42 are multiplied on the tensor cores with FP32
accumulation that is exact over each 512-long K segment, and the segments are
summed in double-float.  The truncation leaves about 35 bits relative to the
largest entry of a block row times the largest entry of a source's vector:
~1e-10 on these operators.  Compared with the exact FP64 operator of the oracle
and with the library's double-float product (~1e-14), on shapes with ragged
row tiles (n_t not a multiple of 128) and ragged column tiles (2S not a
multiple of 48), sources of very different magnitudes and a zero source.
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import discretization as D
from oracle import solver as S

pytestmark = pytest.mark.gpu

CASES = [
    W.small_case(40, 60, 8, 3, medium="grf", seed=11),          # n_t = 56: one ragged row tile
    W.small_case(140, 60, 10, 3, medium="layered", seed=3),     # n_t = 160: two row tiles, K = 320 (5 blocks of 64)
    W.small_case(300, 90, 10, 3, medium="grf", seed=4),         # n_t = 320: K = 640 > one 512-long segment
]


def _rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module", params=range(len(CASES)))
def case(request):
    from paper_1410_5910_gb300 import PT_MIXED_TC, PolarTrace

    wl = CASES[request.param]
    c = wl.c_ext()
    om = wl.omega(c)
    prob = D.make_problem(c, wl.npml, wl.h, om)
    solver = PolarTrace(wl.nx, wl.nz, wl.npml, wl.L, wl.h, om, torch.from_numpy(c).cuda(), pml_C=prob.C,
                        precision=PT_MIXED_TC, max_sources=40, max_krylov=40)
    return wl, prob, solver


def _products(solver, x):
    from paper_1410_5910_gb300 import PT_OPT_RESTART

    xt = torch.from_numpy(x).cuda()
    solver.set_option(PT_OPT_RESTART, 1)
    split = solver.apply("restart", xt).cpu().numpy()
    split2 = solver.apply("restart", xt).cpu().numpy()
    solver.set_option(PT_OPT_RESTART, 0)
    df = solver.apply("restart", xt).cpu().numpy()
    solver.set_option(PT_OPT_RESTART, 1)
    exact = solver.matvec(xt).cpu().numpy()  # dense FP64 blocks
    return split, split2, df, exact


@pytest.mark.parametrize("nsrc", [1, 7, 40])
def test_split_restart_product_matches_fp64(case, nsrc):
    wl, prob, solver = case
    g = np.random.default_rng(nsrc)
    x = g.standard_normal((nsrc, solver.T4, solver.nt)) + 1j * g.standard_normal((nsrc, solver.T4, solver.nt))
    split, split2, df, exact = _products(solver, x)
    assert np.array_equal(split, split2)  # deterministic
    for s in range(nsrc):
        assert _rel(df[s], exact[s]) < 1e-12
        assert _rel(split[s], exact[s]) < 2e-9


def test_split_restart_product_with_uneven_magnitudes_and_a_zero_source(case):
    wl, prob, solver = case
    g = np.random.default_rng(5)
    x = g.standard_normal((6, solver.T4, solver.nt)) + 1j * g.standard_normal((6, solver.T4, solver.nt))
    x[1] *= 1e-30
    x[2] *= 1e25
    x[3] = 0.0
    x[4, : solver.T4 // 2] *= 1e-6  # traces of one source spanning six decades
    split, _, _, exact = _products(solver, x)
    assert np.all(split[3] == 0.0)
    for s in (0, 1, 2, 5):
        assert _rel(split[s], exact[s]) < 2e-9
    # within one source, the small traces carry an absolute error relative to the source's largest entry
    assert np.linalg.norm(split[4] - exact[4]) < 2e-9 * np.linalg.norm(exact[4])


def test_tensor_core_solve_with_split_restarts_reaches_the_oracle(case):
    from paper_1410_5910_gb300 import PT_OPT_RESTART

    wl, prob, solver = case
    solver.set_option(PT_OPT_RESTART, 1)
    pos = [(3, 2), (wl.nx // 2, wl.nz // 2), (wl.nx - 1, wl.nz - 3)]
    f = W.point_sources(wl.nt, wl.Nz, wl.npml, wl.h, pos)
    u, _, its, rel = solver.solve(torch.from_numpy(f).cuda(), tol=1e-7)
    ref = S.global_solve(prob, f)
    un = u.cpu().numpy()
    mask = D.physical_mask(prob, wl.nx, wl.nz)
    for s in range(len(pos)):
        assert rel[s] <= 1e-7
        assert _rel(un[s][mask], ref[s][mask]) < 1e-5
