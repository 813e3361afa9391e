"""Pins of the oracle's discretization (Section 2.1) and layering (Section 2.2).

CPU only.  The free-space check compares with the closed form (i/4) H0(1)(omega r)
from scipy.special, the outgoing Green's function of -Laplace - omega^2 under
the e^{-i omega t} convention that alpha = 1/(1 + i sigma/omega) damps.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla
from scipy.special import hankel1

import workloads as W
from oracle import discretization as D
from oracle import solver as S

from .oracle_cases import case, rel


def test_interior_rows_are_the_plain_five_point_stencil():
    # Section 2.1: away from the PML the operator is (4u - neighbours)/h^2 - omega^2 m u.
    nx, npml, h, om = 20, 5, 1 / 21, 30.0
    m = np.full((nx + 2 * npml, nx + 2 * npml), 0.7)
    H = D.helmholtz_operator(m, npml, h, om, 10.0).tocsr()
    nt = m.shape[1]
    for (q, p) in [(npml, npml), (12, 9), (nt - npml - 1, nt - npml - 1)]:
        row = H.getrow(q * nt + p).toarray().ravel()
        expect = np.zeros_like(row)
        expect[q * nt + p] = 4 / h**2 - om**2 * 0.7
        for dq, dp in [(0, 1), (0, -1), (1, 0), (-1, 0)]:
            expect[(q + dq) * nt + p + dp] = -1 / h**2
        assert np.allclose(row, expect, rtol=0, atol=1e-9 / h**2)


def test_pml_profile_edges_and_dirichlet_distance():
    # sigma vanishes between the edges (n_pml - 1 and n - n_pml) and reaches C/delta at the Dirichlet node.
    n, npml, h, om, C = 30, 6, 0.1, 5.0, 7.0
    pos = np.arange(-1, n + 0.5, 0.5)  # -1 .. n, symmetric about (n-1)/2
    a = D.pml_alpha(pos, n, npml, h, om, C)
    inside = (pos >= npml - 1) & (pos <= n - npml)
    assert np.all(a[inside] == 1.0)
    assert np.all(np.abs(a[~inside]) < 1.0)
    sig_at_dirichlet = ((1 / D.pml_alpha(np.array([-1.0, n]), n, npml, h, om, C) - 1) * om / 1j).real
    assert np.allclose(sig_at_dirichlet, C / (npml * h))
    assert np.allclose(a[::-1], a)  # symmetric profile


def test_global_direct_solve_residual():
    _, prob, _, f, u = case()
    H = D.global_operator(prob)
    assert rel(H @ u.ravel(), f.ravel()) < 1e-12


def _hankel_error(n, omega, src_frac=0.25):
    npml = int(round(0.25 * (n + 1)))  # PML of fixed physical width 0.25
    h = 1.0 / (n + 1)
    nt = n + 2 * npml
    c = np.ones((nt, nt))
    prob = D.make_problem(c, npml, h, omega)
    ps = int(round(src_frac * (n + 1)))
    f = W.point_sources(nt, nt, npml, h, [(ps, ps)])[0]
    u = S.global_solve(prob, f)
    p = np.arange(nt) - npml + 1  # physical 1-based index of each column
    X, Z = np.meshgrid(p * h, p * h)
    r = np.hypot(X - ps * h, Z - ps * h)
    lam = 2 * np.pi / omega
    mask = (r >= 2 * lam) & (X >= 2 * h) & (Z >= 2 * h) & (X <= 1 - 2 * h) & (Z <= 1 - 2 * h)
    exact = 0.25j * hankel1(0, omega * r[mask])
    return np.linalg.norm(u[mask] - exact) / np.linalg.norm(exact)


@pytest.mark.slow
def test_point_source_matches_free_space_hankel_at_second_order():
    omega = 2 * np.pi * 4.0
    errs = [_hankel_error(n, omega) for n in (63, 127, 255)]
    assert errs[-1] < 2e-2
    ratios = [errs[i] / errs[i + 1] for i in range(2)]
    # second order: error / 4 per halving of h (allow pollution and PML reflection)
    assert all(3.0 < q < 5.0 for q in ratios), (errs, ratios)


def test_partition_and_local_rows_match_global():
    wl, prob, off, f, u = case(L=3)
    nc = off.nc
    assert nc[0] == 0 and nc[-1] == prob.Nz and np.all(np.diff(nc) >= 3)
    Hg = D.global_operator(prob).tocsr()
    nt = prob.nt
    for lay in off.layers:
        Hl = D.local_operator(prob, lay).tocsr()
        # rows 1..n of H^l equal the global rows (Section 2.2), couplings included
        for j in (1, 2, lay.n - 1, lay.n):
            rl, rg = lay.row(j), lay.start + j - 1
            loc = Hl[rl * nt : (rl + 1) * nt].toarray()
            glob = Hg[rg * nt : (rg + 1) * nt].toarray()
            # align columns: local row r <-> global row r - pad_top + start
            for dr in (-1, 0, 1):
                a = loc[:, (rl + dr) * nt : (rl + dr + 1) * nt]
                b = glob[:, (rg + dr) * nt : (rg + dr + 1) * nt]
                assert np.allclose(a, b, rtol=1e-14, atol=0)


def test_partition_rejects_interfaces_in_pml():
    with pytest.raises(ValueError):
        D.check_partition(40, 10, np.array([0, 10, 40]))
    with pytest.raises(ValueError):
        D.check_partition(40, 5, np.array([0, 20, 22, 40]))
    D.check_partition(40, 5, np.array([0, 20, 40]))


def test_normal_extension_of_the_model():
    wl, prob, off, f, u = case(medium="grf", seed=7, L=3)
    lay = off.layers[1]
    m = prob.m
    assert np.array_equal(lay.m_local[: lay.pad_top], np.repeat(m[lay.start][None], lay.pad_top, 0))
    assert np.array_equal(lay.m_local[lay.pad_top + lay.n :], np.repeat(m[lay.start + lay.n - 1][None], lay.pad_bot, 0))
    assert np.array_equal(lay.m_local[lay.pad_top : lay.pad_top + lay.n], m[lay.start : lay.start + lay.n])
