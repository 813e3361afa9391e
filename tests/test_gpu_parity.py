"""GPU parity of the CUDA path against the CPU oracle (calls go through the C ABI).

Tolerances: the FP64 path reaches the exact discrete solution up to rounding
(Theorem 1, Proposition 1), so blocks and operator applications are compared
at 1e-10 relative (FP64 with condition numbers of the local problems ~1e4);
volume fields after GMRES at 1e-6 relative L2 over the physical region, the
bound the FP64 mode must meet; the mixed FP32 preconditioner at 1e-5.
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


def _mk(wl, precision=0, max_sources=1, max_krylov=40, gs_iters=2):
    from paper_1410_5910_gb300 import PolarTrace

    c = wl.c_ext()
    om = wl.omega(c)
    prob = D.make_problem(c, wl.npml, wl.h, om)
    solver = PolarTrace(wl.nx, wl.nz, wl.npml, wl.L, wl.h, om, torch.from_numpy(c).cuda(), pml_C=prob.C,
                        precision=precision, max_sources=max_sources, max_krylov=max_krylov, gs_iters=gs_iters)
    return prob, solver


SMALL = [
    W.small_case(40, 60, 8, 3, medium="grf", seed=11),
    W.small_case(37, 45, 6, 4, medium="constant", sources=((5, 30),)),  # ragged n_t, source in layer 2
    W.small_case(50, 23, 5, 2, medium="grf", seed=12, sources=((25, 3),)),  # two layers
]


@pytest.fixture(scope="module", params=range(len(SMALL)))
def small(request):
    wl = SMALL[request.param]
    prob, solver = _mk(wl)
    off = S.precompute(prob, wl.L)
    return wl, prob, solver, off


def test_green_blocks_match_oracle(small):
    wl, prob, solver, off = small
    h = prob.h
    for l, G in enumerate(off.blocks):
        for (j, k), blk in G.items():
            got = solver.block(l, j, k).cpu().numpy()
            assert _rel(got, blk / h) < 1e-10, (l, j, k)


def _rand_vec(solver, seed, S_=1):
    g = np.random.default_rng(seed)
    x = g.standard_normal((S_, solver.T4, solver.nt)) + 1j * g.standard_normal((S_, solver.T4, solver.nt))
    return x


def test_operator_applications_match_oracle(small):
    wl, prob, solver, off = small
    sp_ = off.split
    x = _rand_vec(solver, 1)
    xt = torch.from_numpy(x).cuda()
    assert _rel(solver.matvec(xt).cpu().numpy()[0].ravel(), sp_.PM.apply(x[0].ravel())) < 1e-11
    assert _rel(solver.apply_R(xt).cpu().numpy()[0].ravel(), sp_.apply_R(x[0].ravel())) < 1e-11
    assert _rel(solver.apply_D_inverse(xt).cpu().numpy()[0].ravel(), sp_.solve_D(x[0].ravel())) < 1e-11
    # Algorithm 4 acts on an unpermuted residual in the oracle; the library takes the permuted one
    perm = sp_.perm
    unperm = np.empty_like(x[0])
    unperm[perm] = x[0]
    ref = polarized.gauss_seidel_preconditioner(sp_, unperm.ravel(), 2)
    assert _rel(solver.precond(xt).cpu().numpy()[0].ravel(), ref) < 1e-11


def test_rhs_matches_oracle(small):
    wl, prob, solver, off = small
    f = wl.f()
    got = solver.rhs(torch.from_numpy(f).cuda()).cpu().numpy()[0].ravel()
    ref = polarized.apply_P(S.polarized_rhs(off, f[0]), off.L, prob.nt)
    assert _rel(got, ref) < 1e-11


def test_end_to_end_fp64_matches_global_solve(small):
    wl, prob, solver, off = small
    f = wl.f()
    u_ref = S.global_solve(prob, f[0])
    u, tr, its, rel = solver.solve(torch.from_numpy(f).cuda(), tol=1e-10)
    u = u.cpu().numpy()[0]
    mask = D.physical_mask(prob, wl.nx, wl.nz)
    assert rel[0] <= 1e-10
    assert _rel(u[mask], u_ref[mask]) < 1e-6
    assert _rel(u, u_ref) < 1e-6
    # traces: u_down + u_up equal the global traces (Proposition 1 / Theorem 1)
    T = 2 * (wl.L - 1)
    trn = tr.cpu().numpy()[0]
    assert _rel(trn[:T] + trn[T:], S.global_traces(u_ref, off.nc).reshape(T, -1)) < 1e-6
    # and the oracle's own polarized-traces solve takes the same number of iterations (+-1)
    ores = S.online_solve(off, f[0], tol=1e-10)
    assert abs(ores.iterations - its[0]) <= 1


def test_mixed_fp32_preconditioner_meets_mixed_tolerance(small):
    wl, prob, _, off = small
    _, solver = _mk(wl, precision=1)
    f = wl.f()
    u_ref = S.global_solve(prob, f[0])
    u, tr, its, rel = solver.solve(torch.from_numpy(f).cuda(), tol=1e-9)
    mask = D.physical_mask(prob, wl.nx, wl.nz)
    assert rel[0] <= 1e-9
    # FP32 local solves (FP64 factors rounded to complex64): ~1e-6 on the field
    assert _rel(u.cpu().numpy()[0][mask], u_ref[mask]) < 1e-5
    assert _rel(u.cpu().numpy()[0], u_ref) < 1e-5


@pytest.mark.parametrize("variant,tol_field", [(0, 1e-5), (1, 1e-8), (2, 1e-5), (3, 1e-5), (4, 1e-5)])
def test_mixed_local_solve_variants_match_oracle(small, variant, tol_field):
    """FP32 local solves on clusters of 4 or 8 CTAs, on one CTA, or chunked along x (one CTA per chunk, boundary
    values propagated between chunks), and double-float ones, on a point source and on a source that excites every
    layer."""
    from paper_1410_5910_gb300 import PT_OPT_LOCAL_SOLVE

    wl, prob, _, off = small
    _, solver = _mk(wl, precision=1, max_sources=2)
    solver.set_option(PT_OPT_LOCAL_SOLVE, variant)
    f = np.concatenate([wl.f(), W.random_sources(wl.nt, wl.Nz, wl.npml, wl.nx, wl.nz, 9, 1)])
    u, tr, its, rel = solver.solve(torch.from_numpy(f).cuda(), tol=1e-10)
    for s in range(2):
        assert rel[s] <= 1e-10
        assert _rel(u.cpu().numpy()[s], S.global_solve(prob, f[s])) < tol_field


@pytest.mark.parametrize("nsrc", [1, 3])
def test_one_launch_sweeps_match_per_step_sweeps_and_oracle(small, nsrc):
    """The FP32 preconditioner with all sweep steps in one cooperative launch (default) against one launch
    per step (the same products in the same order) and against Algorithm 4 of the oracle; the FP16 one
    (PT_OPT_PRECOND_FP16) against the oracle at its own accuracy."""
    from paper_1410_5910_gb300 import PT_OPT_PRECOND_FP16, PT_OPT_SWEEP

    wl, prob, _, off = small
    _, solver = _mk(wl, precision=1, max_sources=nsrc)
    x = _rand_vec(solver, 5, nsrc)
    xt = torch.from_numpy(x).cuda()
    solver.set_option(PT_OPT_PRECOND_FP16, 1)
    half = solver.precond(xt).cpu().numpy()
    solver.set_option(PT_OPT_PRECOND_FP16, 0)
    fused = solver.precond(xt).cpu().numpy()
    solver.set_option(PT_OPT_SWEEP, 1)
    stepped = solver.precond(xt).cpu().numpy()
    sp_ = off.split
    for q in range(nsrc):
        assert _rel(fused[q], stepped[q]) < 1e-12
        unperm = np.empty_like(x[q])
        unperm[sp_.perm] = x[q]
        ref = polarized.gauss_seidel_preconditioner(sp_, unperm.ravel(), 2)
        assert _rel(fused[q].ravel(), ref) < 1e-5
        assert _rel(half[q].ravel(), ref) < 1e-2
    # and a whole solve with each
    f = wl.f()
    solver.set_option(PT_OPT_SWEEP, 0)
    u0, _, its0, rel0 = solver.solve(torch.from_numpy(f).cuda(), tol=1e-10)
    solver.set_option(PT_OPT_SWEEP, 1)
    u1, _, its1, rel1 = solver.solve(torch.from_numpy(f).cuda(), tol=1e-10)
    assert its0[0] == its1[0] and rel0[0] <= 1e-10
    assert _rel(u0.cpu().numpy(), u1.cpu().numpy()) < 1e-9


@pytest.mark.parametrize("nsrc", [1, 3])
def test_mixed_working_operators_match_oracle(small, nsrc):
    """The operators PT_MIXED_FP32 iterates with: double-float P M (~1e-14); R and D^{-1} with the FP32 blocks
    (default, ~1e-7) and with the row-scaled FP16 blocks (option, ~1e-4), against the oracle's FP64 operators."""
    from paper_1410_5910_gb300 import PT_OPT_PRECOND_FP16

    wl, prob, _, off = small
    _, solver = _mk(wl, precision=1, max_sources=nsrc)
    x = _rand_vec(solver, 21, nsrc)
    xt = torch.from_numpy(x).cuda()
    sp_ = off.split
    solver.set_option(PT_OPT_PRECOND_FP16, 1)
    half = {w: solver.apply(w, xt, working=True).cpu().numpy() for w in ("R", "Dinv")}
    solver.set_option(PT_OPT_PRECOND_FP16, 0)
    got = {w: solver.apply(w, xt, working=True).cpu().numpy() for w in ("matvec", "R", "Dinv")}
    for q in range(nsrc):
        xs = x[q].ravel()
        assert _rel(got["matvec"][q].ravel(), sp_.PM.apply(xs)) < 1e-12
        assert _rel(got["R"][q].ravel(), sp_.apply_R(xs)) < 2e-6
        assert _rel(got["Dinv"][q].ravel(), sp_.solve_D(xs)) < 2e-6
        assert _rel(half["R"][q].ravel(), sp_.apply_R(xs)) < 5e-3
        assert _rel(half["Dinv"][q].ravel(), sp_.solve_D(xs)) < 1e-2


@pytest.mark.parametrize("sources", [((100, 60),), ((7, 3), (190, 110), (60, 95))])
def test_chunked_local_solves_match_oracle_medium(sources):
    """Chunked local solves (13 chunks of 16-17 columns per layer) on a 200 x 120 grid: point sources near the corners
    and in the middle.  The solve runs both chunked local solves (the interface right-hand side and the
    reconstruction); each solution against the oracle's global sparse solve and against the same solve with the
    clustered local solves (same GMRES iteration count: the right-hand sides agree)."""
    from paper_1410_5910_gb300 import PT_OPT_LOCAL_SOLVE

    wl = W.small_case(200, 120, 10, 4, medium="grf", seed=5, sources=sources)
    prob, solver = _mk(wl, precision=1, max_sources=len(sources))
    f = wl.f()
    ft = torch.from_numpy(f).cuda()
    solver.set_option(PT_OPT_LOCAL_SOLVE, 4)
    u4, _, its4, rel4 = solver.solve(ft, tol=1e-10)
    solver.set_option(PT_OPT_LOCAL_SOLVE, 0)
    u0, _, its0, rel0 = solver.solve(ft, tol=1e-10)
    ref = S.global_solve(prob, f)
    for q in range(len(sources)):
        assert rel4[q] <= 1e-10 and its4[q] == its0[q]
        assert _rel(u4[q].cpu().numpy(), ref[q]) < 1e-5
        assert _rel(u4[q].cpu().numpy(), u0[q].cpu().numpy()) < 1e-5


@pytest.mark.parametrize("tol", [1e-7, 1e-10])
def test_relaxed_matvecs_keep_the_tolerance(tol):
    """Inexact Krylov relaxation of the mixed form (FP32 matvecs once the residual estimate is below 1e4 tol ||b||)
    against double-float matvecs throughout: both reach tol (the restart residual is double-float), the same
    iteration count up to one, some matvecs relaxed, the fields within the FP32 local-solve accuracy of each other
    and of the oracle."""
    from paper_1410_5910_gb300 import PT_OPT_RELAX

    wl = W.small_case(200, 120, 10, 4, medium="grf", seed=7, sources=((100, 60), (30, 100)))
    prob, solver = _mk(wl, precision=1, max_sources=2)
    ft = torch.from_numpy(wl.f()).cuda()
    u1, _, its1, rel1 = solver.solve(ft, tol=tol)
    n_relaxed = solver.last_solve_relaxed()
    solver.set_option(PT_OPT_RELAX, 0)
    u0, _, its0, rel0 = solver.solve(ft, tol=tol)
    assert solver.last_solve_relaxed() == 0 and n_relaxed >= 1
    ref = S.global_solve(prob, wl.f())
    for q in range(2):
        assert rel1[q] <= tol and rel0[q] <= tol
        assert abs(its1[q] - its0[q]) <= 1
        assert _rel(u1[q].cpu().numpy(), u0[q].cpu().numpy()) < 1e-5
        assert _rel(u1[q].cpu().numpy(), ref[q]) < max(1e-5, 10 * tol)


def test_fp16_preconditioner_keeps_iterations_and_tolerance():
    """The FP16 preconditioner blocks (option) against the FP32 ones on a 200 x 120 grid with 13-17 column chunks:
    both solves reach the tolerance, with at most two more iterations, and the same field."""
    from paper_1410_5910_gb300 import PT_OPT_PRECOND_FP16

    wl = W.small_case(200, 120, 10, 4, medium="grf", seed=9, sources=((50, 40), (150, 90)))
    prob, solver = _mk(wl, precision=1, max_sources=2)
    ft = torch.from_numpy(wl.f()).cuda()
    solver.set_option(PT_OPT_PRECOND_FP16, 1)
    u16, _, its16, rel16 = solver.solve(ft, tol=1e-8)
    solver.set_option(PT_OPT_PRECOND_FP16, 0)
    u32, _, its32, rel32 = solver.solve(ft, tol=1e-8)
    ref = S.global_solve(prob, wl.f())
    for q in range(2):
        assert rel16[q] <= 1e-8 and rel32[q] <= 1e-8
        assert its16[q] <= its32[q] + 2
        assert _rel(u16[q].cpu().numpy(), u32[q].cpu().numpy()) < 1e-5
        assert _rel(u16[q].cpu().numpy(), ref[q]) < 1e-5


def test_batched_sources_equal_single_solves():
    wl = W.small_case(40, 60, 8, 3, medium="grf", seed=11)
    prob, solver = _mk(wl, max_sources=3)
    f = W.point_sources(wl.nt, wl.Nz, wl.npml, wl.h, [(5, 5), (20, 30), (39, 58)])
    ub, _, itb, relb = solver.solve(torch.from_numpy(f).cuda(), tol=1e-10)
    ref = S.global_solve(prob, f)
    for s in range(3):
        u1, _, it1, rel1 = solver.solve(torch.from_numpy(f[s : s + 1]).cuda(), tol=1e-10)
        assert _rel(ub[s].cpu().numpy(), u1[0].cpu().numpy()) < 1e-9
        assert _rel(ub[s].cpu().numpy(), ref[s]) < 1e-6


def test_random_sources_everywhere():
    wl = W.small_case(40, 60, 8, 3, medium="grf", seed=11)
    prob, solver = _mk(wl, max_sources=2)
    f = W.random_sources(wl.nt, wl.Nz, wl.npml, wl.nx, wl.nz, seed=3, count=2)
    u, _, its, rel = solver.solve(torch.from_numpy(f).cuda(), tol=1e-10)
    ref = S.global_solve(prob, f)
    assert _rel(u.cpu().numpy(), ref) < 1e-6


def test_zero_source_gives_zero_field():
    wl = W.small_case(40, 60, 8, 3, medium="grf", seed=11)
    prob, solver = _mk(wl)
    f = torch.zeros((1, wl.Nz, wl.nt), dtype=torch.complex128, device="cuda")
    u, tr, its, rel = solver.solve(f, tol=1e-10)
    assert its[0] == 0 and float(u.abs().max()) == 0.0


def test_host_entry_point_matches_device_entry_point():
    wl = W.small_case(40, 60, 8, 3, medium="grf", seed=11)
    prob, solver = _mk(wl)
    f = wl.f()
    u_dev, _, its_d, _ = solver.solve(torch.from_numpy(f).cuda(), tol=1e-10)
    f_h = torch.from_numpy(f).pin_memory()
    u_h = torch.empty_like(f_h).pin_memory()
    its_h, rel_h = solver.solve_host(f_h, u_h, tol=1e-10)
    assert its_h == its_d
    assert _rel(u_h.numpy(), u_dev.cpu().numpy()) < 1e-13


def test_invalid_medium_is_rejected():
    from paper_1410_5910_gb300 import PolarTrace, PolarTraceError

    wl = W.small_case(40, 60, 8, 3)
    c = wl.c_ext()
    c[10, 10] = -1.0
    with pytest.raises(PolarTraceError, match="NUMERIC"):
        PolarTrace(wl.nx, wl.nz, wl.npml, wl.L, wl.h, 10.0, torch.from_numpy(c).cuda())
    c[10, 10] = np.nan  # pml_C given explicitly so that the medium check, not the argument check, fires
    with pytest.raises(PolarTraceError, match="NUMERIC"):
        PolarTrace(wl.nx, wl.nz, wl.npml, wl.L, wl.h, 10.0, torch.from_numpy(c).cuda(), pml_C=20.0)


def test_not_converged_reports_status():
    from paper_1410_5910_gb300 import PolarTraceError

    wl = W.small_case(40, 60, 8, 3, medium="grf", seed=11)
    prob, solver = _mk(wl)
    f = torch.from_numpy(wl.f()).cuda()
    with pytest.raises(PolarTraceError, match="NOT_CONVERGED"):
        solver.solve(f, tol=1e-14, max_it=1)
    u, _, its, rel = solver.solve(f, tol=1e-14, max_it=1, allow_not_converged=True)
    assert its[0] == 1 and rel[0] > 1e-14


@pytest.mark.slow
def test_constant_128_workload_matches_global_solve():
    wl = W.CONSTANT_128
    prob, solver = _mk(wl)
    f = wl.f()
    u, tr, its, rel = solver.solve(torch.from_numpy(f).cuda(), tol=wl.tol)
    u_ref = S.global_solve(prob, f[0])
    mask = D.physical_mask(prob, wl.nx, wl.nz)
    assert rel[0] <= wl.tol
    assert _rel(u.cpu().numpy()[0][mask], u_ref[mask]) < 1e-6
    assert its[0] <= 10
