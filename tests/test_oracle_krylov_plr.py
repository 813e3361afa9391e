"""Pins of the oracle's GMRES (Section 4.2), PLR compression (Section 5.1) and end-to-end solve.

CPU only.  GMRES is pinned by brute force: after k steps its iterate must be
the minimiser of the residual over the k-dimensional Krylov space, computed
here by an explicit least-squares solve, and it must agree with SciPy's GMRES.
PLR is pinned by exactly low-rank matrices and by the error bound the
truncation implies.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import krylov, plr, polarized
from oracle import solver as S

from .oracle_cases import case, rel


def _rand(n, seed):
    g = np.random.default_rng(seed)
    return g.standard_normal((n, n)) + 1j * g.standard_normal((n, n)), g.standard_normal(n) + 1j * g.standard_normal(n)


@pytest.mark.parametrize("k", [1, 3, 6])
def test_gmres_iterate_minimises_residual_over_krylov_space(k):
    n = 40
    A, b = _rand(n, 0)
    A = A + 8 * np.eye(n)
    x, its, hist = krylov.gmres_left(lambda v: A @ v, b, lambda v: v, tol=1e-30, max_it=k)
    assert its == k
    K = np.stack([np.linalg.matrix_power(A, i) @ b for i in range(k)], axis=1)
    Q, _ = np.linalg.qr(K)
    y, *_ = np.linalg.lstsq(A @ Q, b, rcond=None)
    assert rel(x, Q @ y) < 1e-10
    assert abs(hist[-1] - np.linalg.norm(b - A @ x)) < 1e-10 * np.linalg.norm(b)


@pytest.mark.parametrize("k", [2, 5])
def test_right_preconditioned_iterate_minimises_over_preconditioned_space(k):
    n = 30
    A, b = _rand(n, 1)
    A = A + 6 * np.eye(n)
    Mi, _ = _rand(n, 2)
    Mi = np.eye(n) + 0.05 * Mi
    x, its, rel_true, hist = krylov.fgmres_right(lambda v: A @ v, b, lambda v: Mi @ v, tol=1e-30, max_it=k, max_cycles=1)
    AM = A @ Mi
    K = np.stack([np.linalg.matrix_power(AM, i) @ b for i in range(k)], axis=1)
    Q, _ = np.linalg.qr(K)
    y, *_ = np.linalg.lstsq(AM @ Q, b, rcond=None)
    assert rel(x, Mi @ (Q @ y)) < 1e-9


def test_gmres_agrees_with_scipy_and_direct_solution():
    n = 60
    A, b = _rand(n, 3)
    A = A + 12 * np.eye(n)
    x, its, hist = krylov.gmres_left(lambda v: A @ v, b, lambda v: v, tol=1e-12, max_it=n)
    xs, info = spla.gmres(A, b, rtol=1e-12, restart=n, maxiter=n)
    xd = np.linalg.solve(A, b)
    assert info == 0
    assert rel(x, xd) < 1e-10 and rel(xs, xd) < 1e-9


@pytest.mark.parametrize("kw", [dict(), dict(medium="grf", seed=3, L=4, nz=40)])
@pytest.mark.parametrize("form", ["right", "left"])
def test_preconditioned_gmres_on_polarized_system_reaches_global_solution(kw, form):
    wl, prob, off, f, u = case(**kw)
    res = S.online_solve(off, f, tol=1e-12, form=form)
    assert rel(res.u, u) < 1e-10
    assert res.true_relres < 1e-11
    # the paper observes a handful of iterations for smooth media (Section 7)
    assert res.iterations <= 10


def test_gauss_seidel_preconditioner_equals_its_dense_formula():
    # Algorithm 4 with n_it = 2: D^{-1}(P f - R D^{-1} P f)
    wl, prob, off, f, u = case(medium="grf", seed=3, L=4, nz=40)
    g = np.random.default_rng(4)
    v = g.standard_normal(off.system.nrows * prob.nt) + 1j * g.standard_normal(off.system.nrows * prob.nt)
    Dd = off.split.PM.dense(off.split.in_D)
    Rd = off.split.PM.dense(off.split.in_R)
    Pv = polarized.apply_P(v, off.L, prob.nt)
    u1 = np.linalg.solve(Dd, Pv)
    u2 = np.linalg.solve(Dd, Pv - Rd @ u1)
    assert rel(polarized.gauss_seidel_preconditioner(off.split, v, 2), u2) < 1e-11
    assert rel(polarized.gauss_seidel_preconditioner(off.split, v, 1), u1) < 1e-11


# --- PLR ---------------------------------------------------------------------


def test_exactly_low_rank_matrix_is_one_leaf():
    g = np.random.default_rng(5)
    m, n, k = 96, 80, 6
    A = (g.standard_normal((m, k)) + 1j * g.standard_normal((m, k))) @ (g.standard_normal((k, n)) + 1j * g.standard_normal((k, n)))
    H = plr.compress(A, r_max=10, eps=1e-9)
    assert H.kind == "c" and H.US.shape == (m, k) and H.Vt.shape == (k, n)
    assert rel(plr.to_dense(H), A) < 1e-12


def test_plr_error_bound_and_recursive_equals_flattened_product():
    # a smooth oscillatory kernel: low rank away from the diagonal, full rank near it
    n = 128
    x = np.arange(n) / n
    A = np.exp(1j * 40 * np.abs(x[:, None] - x[None, :])) / (1 + 30 * np.abs(x[:, None] - x[None, :]))
    eps, rmax = 1e-9, 8
    H = plr.compress(A, rmax, eps)
    lv = plr.leaves(H)
    assert len(lv) > 1
    assert plr.compressed_entries(H) < A.size
    s1 = np.linalg.norm(A, 2)
    err = np.linalg.norm(plr.to_dense(H) - A, 2)
    # each leaf drops singular values below eps * sigma_1
    assert err <= eps * s1 * len(lv) * 10
    g = np.random.default_rng(6)
    X = g.standard_normal((n, 3)) + 1j * g.standard_normal((n, 3))
    assert rel(plr.matvec(H, X), plr.to_dense(H) @ X) < 1e-13
    assert rel(plr.leaf_matvec(lv, n, X), plr.to_dense(H) @ X) < 1e-13
    # leaves tile the matrix exactly once
    cover = np.zeros((n, n), dtype=int)
    for lf in lv:
        cover[lf.rows[0] : lf.rows[1], lf.cols[0] : lf.cols[1]] += 1
    assert np.all(cover == 1)


def test_plr_split_is_ceil_half_and_small_blocks_are_leaves():
    g = np.random.default_rng(7)
    A = g.standard_normal((21, 19)) + 1j * g.standard_normal((21, 19))
    H = plr.compress(A, r_max=4, eps=1e-12)
    assert H.kind == "h"
    assert H.children[0].rows == (0, 11) and H.children[0].cols == (0, 10)
    for lf in plr.leaves(H):
        assert min(lf.rows[1] - lf.rows[0], lf.cols[1] - lf.cols[0]) <= 4 or lf.US is not None
    assert rel(plr.to_dense(H), A) < 1e-12


def test_plr_compressed_green_blocks_keep_the_solution():
    # compress every interface block, then solve with the compressed operator
    wl, prob, off, f, u = case(medium="grf", seed=3, L=4, nz=40, nx=40)
    blocks_c = []
    for G in off.blocks:
        blocks_c.append({k: plr.to_dense(plr.compress(v, 6, 1e-10)) for k, v in G.items()})
    system = polarized.polarized_jump_system(blocks_c, off.ns, prob.h, prob.nt)
    b = S.polarized_rhs(off, f)
    x = np.linalg.solve(system.dense(), b)
    xd = np.linalg.solve(off.system.dense(), b)
    assert rel(x, xd) < 1e-6
