"""Pins of the oracle's Green's matrices and integral / polarized systems (Sections 2.3-4.1).

CPU only.  Every check is an identity the paper proves (Lemmas 1-4, Theorem 1,
Remark 1, the spectral statement of Section 4.2) or a brute-force comparison
with the global sparse direct solve; they hold to round-off on any grid, so a
dropped term, a wrong sign or a transposed block fails them.
"""
import numpy as np
import pytest

from oracle import green, integral, polarized
from oracle import solver as S

from .oracle_cases import case, rel

CASES = [
    dict(),
    dict(medium="grf", seed=3, L=4, nz=40),
    dict(medium="grf", seed=5, L=2, nx=20, nz=16, npml=4),
]


@pytest.mark.parametrize("kw", CASES)
def test_lemma1_grf_reproduces_global_solution_and_vanishes_outside(kw):
    wl, prob, off, f, u = case(**kw)
    nt = prob.nt
    for l, (lay, s) in enumerate(zip(off.layers, off.solvers)):
        tr = {}
        if l > 0:
            tr[0], tr[1] = u[lay.start - 1], u[lay.start]
        if l < off.L - 1:
            e = lay.start + lay.n
            tr[lay.n], tr[lay.n + 1] = u[e - 1], u[e]
        v = green.reconstruct_layer(s, f, tr)
        inside = v[lay.pad_top : lay.pad_top + lay.n]
        assert rel(inside, u[lay.start : lay.start + lay.n]) < 1e-11
        outside = np.concatenate([v[: lay.pad_top], v[lay.pad_top + lay.n :]])
        if outside.size:
            assert np.linalg.norm(outside) < 1e-11 * np.linalg.norm(u)
    assert nt == u.shape[1]


def test_definition2_matrix_form_equals_definition():
    wl, prob, off, f, u = case(medium="grf", seed=3, L=4, nz=40)
    rng = np.random.default_rng(0)
    G, n, h, nt = off.blocks[1], off.ns[1], prob.h, prob.nt
    v = [rng.standard_normal(nt) + 1j * rng.standard_normal(nt) for _ in range(4)]
    for j in (0, 1, n, n + 1):
        dt = integral.down_terms(G, j, h, (0, 1))
        mat = dt[0][1] @ v[0] + dt[1][1] @ v[1]
        assert rel(mat, green.incomplete_green_down(G, j, v[0], v[1], h)) < 1e-13
        ut = integral.up_terms(G, j, n, h, (0, 1))
        mat = ut[0][1] @ v[2] + ut[1][1] @ v[3]
        assert rel(mat, green.incomplete_green_up(G, j, n, v[2], v[3], h)) < 1e-13


def test_green_blocks_are_columns_of_the_local_inverse():
    # Definition 1: H^l G = delta with delta = 1/h^2, G(z_j,z_k) = h * (H^l)^{-1}/h^2 restricted.
    wl, prob, off, f, u = case()
    s, lay = off.solvers[1], off.layers[1]
    n = lay.n
    col = 7
    sampled = green.green_column(s, (0, 1, n, n + 1), n, col)
    for j in (0, 1, n, n + 1):
        assert rel(sampled[j], off.blocks[1][(j, n)][:, col]) < 1e-13
    # apply H^l to the full local column and check the discrete delta
    rhs = np.zeros(lay.nloc * prob.nt, dtype=complex)
    rhs[lay.row(n) * prob.nt + col] = 1.0
    x = s.solve(rhs[:, None])[:, 0] / prob.h**2  # G on the grid, delta scaled
    hx = s.H @ x
    expect = np.zeros_like(hx)
    expect[lay.row(n) * prob.nt + col] = 1 / prob.h**2
    assert rel(hx, expect) < 1e-12


@pytest.mark.parametrize("kw", CASES[:2])
def test_lemma4_extrapolator_identities(kw):
    wl, prob, off, f, u = case(**kw)
    h = prob.h
    for l in range(off.L - 1):
        Gl, n = off.blocks[l], off.ns[l]
        Gn = off.blocks[l + 1]
        nn = off.ns[l + 1]
        Eup = polarized.extrapolator_up(Gn)
        targets_up = [1] + ([nn, nn + 1] if l + 1 < off.L - 1 else [])
        for j in targets_up:
            assert rel(Eup @ Gn[(1, j)], Gn[(0, j)]) < 1e-9
        assert rel(Eup @ Gn[(1, 0)], Gn[(0, 0)] - h * Eup) < 1e-9
        Edn = polarized.extrapolator_down(Gl, n)
        targets_dn = [n] + ([0, 1] if l > 0 else [])
        for j in targets_dn:
            assert rel(Edn @ Gl[(n, j)], Gl[(n + 1, j)]) < 1e-9
        assert rel(Edn @ Gl[(n, n + 1)], Gl[(n + 1, n + 1)] - h * Edn) < 1e-9


@pytest.mark.parametrize("kw", CASES)
def test_theorem1_integral_system_gives_global_traces(kw):
    wl, prob, off, f, u = case(**kw)
    nt = prob.nt
    M = integral.integral_system(off.blocks, off.ns, prob.h, nt)
    nw = S.newton_traces(off, f)
    fu = integral.integral_rhs(nw, off.ns, nt)
    tr = np.linalg.solve(M.dense(), -fu)
    gt = S.global_traces(u, off.nc)
    assert rel(tr, gt) < 1e-10
    # Remark 1 / Lemma 2: the same traces satisfy the M_0 system
    M0 = integral.integral_system_outside(off.blocks, off.ns, prob.h, nt)
    f0 = integral.integral_rhs(nw, off.ns, nt, outside=True)
    assert rel(M0.apply(gt), -f0) < 1e-10


@pytest.mark.parametrize("kw", CASES)
def test_polarized_system_solution_is_polarized_and_sums_to_traces(kw):
    wl, prob, off, f, u = case(**kw)
    nt, h, L = prob.nt, prob.h, off.L
    T = 2 * (L - 1)
    b = S.polarized_rhs(off, f)
    x = np.linalg.solve(off.system.dense(), b)
    gt = S.global_traces(u, off.nc)
    assert rel(polarized.collapse(x, L, nt), gt) < 1e-10
    X = x.reshape(2 * T, nt)
    dn, up = X[:T], X[T:]
    scale = np.linalg.norm(gt)
    for i in range(L - 1):
        # Definition 5: annihilation relations at interface i
        Gn = off.blocks[i + 1]
        a = green.incomplete_green_down(Gn, 1, up[2 * i], up[2 * i + 1], h)
        assert np.linalg.norm(a) < 1e-9 * scale
        Gl, n = off.blocks[i], off.ns[i]
        a = green.incomplete_green_up(Gl, n, n, dn[2 * i], dn[2 * i + 1], h)
        assert np.linalg.norm(a) < 1e-9 * scale
        # Lemma 3: extrapolators reproduce the polarized traces
        assert np.linalg.norm(polarized.extrapolator_up(Gn) @ up[2 * i + 1] - up[2 * i]) < 1e-8 * scale
        assert np.linalg.norm(polarized.extrapolator_down(Gl, n) @ dn[2 * i] - dn[2 * i + 1]) < 1e-8 * scale


@pytest.mark.parametrize("kw", CASES[:2])
def test_splitting_structure_and_half_of_the_spectrum_is_one(kw):
    wl, prob, off, f, u = case(**kw)
    nt, L = prob.nt, off.L
    sp_ = off.split
    assert sorted(sp_.perm.tolist()) == list(range(4 * (L - 1)))
    PM = sp_.PM.dense()
    Dd = sp_.PM.dense(sp_.in_D)
    Rd = sp_.PM.dense(sp_.in_R)
    assert np.allclose(PM, Dd + Rd)
    N = PM.shape[0]
    half = N // 2
    # D_down lower and D_up upper block triangular with -I diagonal blocks (Section 3.5)
    assert np.allclose(np.diag(Dd), -1)
    for r in range(half // nt):
        for c in range(r + 1, half // nt):
            assert not np.any(Dd[r * nt : (r + 1) * nt, c * nt : (c + 1) * nt])
            assert not np.any(Dd[half + c * nt : half + (c + 1) * nt, half + r * nt : half + (r + 1) * nt])
    assert not np.any(Dd[:half, half:]) and not np.any(Dd[half:, :half])
    # Section 4.2: eigenvalues of D^{-1} P M are 1 (half of them) and 1 +- sqrt(mu)
    ev = np.linalg.eigvals(np.linalg.solve(Dd, PM))
    assert np.sum(np.abs(ev - 1) < 1e-7) >= half
    Ud, Ld = Rd[:half, half:], Rd[half:, :half]
    Ddn, Dup = Dd[:half, :half], Dd[half:, half:]
    mu = np.linalg.eigvals(np.linalg.solve(Dup, Ld) @ np.linalg.solve(Ddn, Ud))
    # det(D^{-1}PM - lambda) = det((1 - lambda)^2 I - W): the roots are 1 +- sqrt(mu)
    # (compare on the (1 - lambda)^2 scale: the square root amplifies the rounding of mu ~ 0)
    d = np.abs((1 - ev)[:, None] ** 2 - mu[None, :])
    tol = 1e-9 * max(1.0, np.abs(mu).max())
    assert d.min(axis=1).max() < tol and d.min(axis=0).max() < tol


def test_block_back_substitution_matches_dense_solve():
    wl, prob, off, f, u = case(medium="grf", seed=3, L=4, nz=40)
    rng = np.random.default_rng(1)
    b = rng.standard_normal(off.split.PM.nrows * prob.nt) + 1j * rng.standard_normal(off.split.PM.nrows * prob.nt)
    Dd = off.split.PM.dense(off.split.in_D)
    assert rel(off.split.solve_D(b), np.linalg.solve(Dd, b)) < 1e-11


def test_polarization_invariant_constant_medium():
    # A source in the top layer radiates only downward below it: the up-going
    # traces under it are PML reflections only, and shrink as the PML thickens.
    ratios = []
    for npml in (4, 8, 16):
        wl, prob, off, f, u = case(nx=24, nz=36, npml=npml, L=3, src=(12, 3))
        x = np.linalg.solve(off.system.dense(), S.polarized_rhs(off, f))
        T = 2 * (off.L - 1)
        X = x.reshape(2 * T, prob.nt)
        # interfaces strictly below the source layer
        dn, up = X[:T][2:], X[T:][2:]
        ratios.append(np.linalg.norm(up) / np.linalg.norm(dn))
    assert ratios[0] < 0.1
    assert ratios[2] < ratios[0]


def test_gauss_seidel_iteration_converges_to_direct_solution():
    wl, prob, off, f, u = case(medium="grf", seed=3, L=4, nz=40)
    b = S.polarized_rhs(off, f)
    x, its = polarized.gauss_seidel_iteration(off.split, b, tol=1e-12, max_it=200)
    xd = np.linalg.solve(off.system.dense(), b)
    assert rel(x, xd) < 1e-9
    assert its < 200
