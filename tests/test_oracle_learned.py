"""Pins of the learned-correction oracle (oracle/learned.py), CPU only.

The network is not in the paper, so its pins are mathematical: the exact
gradient against central finite differences, the first layer against
scipy's cross-correlation, the GELU form against the erf-based GELU, the
feature maps against a hand-placed entry, and the additive correction inside
flexible GMRES (a perfect correction K^{-1} + N = M^{-1} converges in one
iteration; a zero network changes nothing).
"""
import numpy as np
import pytest
import scipy.signal
import scipy.special

from oracle import krylov, learned, polarized
from oracle import solver as S

from .oracle_cases import case, rel


def _theta(width, k1, seed, scale=0.3):
    g = np.random.default_rng(seed)
    return scale * g.standard_normal(learned.nparams(width, k1))


def test_gradient_matches_central_differences_small_width():
    width, k1 = 6, 3
    g = np.random.default_rng(0)
    X = g.standard_normal((3, learned.CIN, 9))
    T = g.standard_normal((3, learned.CIN, 9))
    th = _theta(width, k1, 1)
    _, grad = learned.loss_and_grad(th, X, T, width, k1)
    eps = 1e-6
    fd = np.empty_like(th)
    for i in range(th.size):
        e = np.zeros_like(th)
        e[i] = eps
        fd[i] = (learned.loss(th + e, X, T, width, k1) - learned.loss(th - e, X, T, width, k1)) / (2 * eps)
    assert np.max(np.abs(fd - grad)) <= 1e-6 * np.max(np.abs(grad))


def test_gradient_matches_central_differences_full_width_sample():
    g = np.random.default_rng(2)
    X = g.standard_normal((2, learned.CIN, 12))
    T = g.standard_normal((2, learned.CIN, 12))
    th = _theta(learned.WIDTH, learned.K1, 3, scale=0.08)
    _, grad = learned.loss_and_grad(th, X, T)
    # a few parameters of every tensor
    offs, off = [], 0
    for _, shp in learned.shapes():
        n = int(np.prod(shp))
        offs += list(off + g.choice(n, size=6, replace=False))
        off += n
    eps = 1e-6
    for i in offs:
        e = np.zeros_like(th)
        e[i] = eps
        fd = (learned.loss(th + e, X, T) - learned.loss(th - e, X, T)) / (2 * eps)
        assert abs(fd - grad[i]) <= 1e-6 * np.max(np.abs(grad)) + 1e-7 * abs(grad[i])


def test_first_layer_is_scipy_cross_correlation():
    g = np.random.default_rng(5)
    W1 = g.standard_normal((4, learned.CIN, 7))
    b1 = g.standard_normal(4)
    X = g.standard_normal((2, learned.CIN, 15))
    h = learned.conv1(W1, b1, X)
    for s in range(2):
        for o in range(4):
            ref = b1[o] + sum(scipy.signal.correlate(X[s, c], W1[o, c], mode="same") for c in range(learned.CIN))
            assert np.allclose(h[s, o], ref, atol=1e-12)
    # a kernel with one non-zero tap at k shifts the input by k - 3
    W1 = np.zeros((1, learned.CIN, 7))
    W1[0, 2, 5] = 1.0
    h = learned.conv1(W1, np.zeros(1), X)
    assert np.allclose(h[0, 0, :-2], X[0, 2, 2:]) and np.allclose(h[0, 0, -2:], 0.0)


def test_gelu_tanh_form_and_its_derivative():
    x = np.linspace(-6, 6, 2001)
    exact = 0.5 * x * (1 + scipy.special.erf(x / np.sqrt(2)))
    assert np.max(np.abs(learned.gelu(x) - exact)) < 1e-3
    assert learned.gelu(0.0) == 0.0
    fd = (learned.gelu(x + 1e-6) - learned.gelu(x - 1e-6)) / 2e-6
    assert np.max(np.abs(fd - learned.gelu_grad(x))) < 1e-8


def test_features_place_each_trace_row_of_each_interface():
    L, nt = 4, 5
    T = 2 * (L - 1)
    v = np.zeros((2 * T, nt), dtype=np.complex128)
    v[T + 2 * 1 + 1, 3] = 2.0 - 7.0j  # up-going row 1 of interface 1
    X = learned.features(v, L)
    nz = np.argwhere(X != 0)
    assert sorted(map(tuple, nz)) == [(1, 6, 3), (1, 7, 3)]
    assert X[1, 6, 3] == 2.0 and X[1, 7, 3] == -7.0
    g = np.random.default_rng(1)
    w = g.standard_normal((2 * T, nt)) + 1j * g.standard_normal((2 * T, nt))
    assert np.array_equal(learned.unfeatures(learned.features(w, L), L), w)


def test_additive_correction_in_flexible_gmres():
    wl, prob, off, f, u = case(medium="grf", seed=3, L=4, nz=40)
    b = S.polarized_rhs(off, f)
    A = off.system.apply
    Md = off.system.dense()
    nt = prob.nt
    K = lambda v: polarized.gauss_seidel_preconditioner(off.split, v, 2)  # noqa: E731
    # a perfect network returns the defect M^{-1} v - K^{-1} v: one iteration
    perfect = lambda v: K(v) + (np.linalg.solve(Md, v) - K(v))  # noqa: E731
    x, its, relres, _ = krylov.fgmres_right(A, b, perfect, 1e-10, 20)
    assert its == 1 and relres < 1e-10
    # training pairs encode exactly that defect: K^{-1} r + RMS(r) N*(P r / RMS(r)) = e
    g = np.random.default_rng(7)
    e = (g.standard_normal(b.size) + 1j * g.standard_normal(b.size)).reshape(-1, nt)
    r = A(e.ravel()).reshape(-1, nt)
    Xin, Tout = learned.training_pair(off.split, r, e, off.L)
    back = K(r.ravel()).reshape(-1, nt) + learned.rms(r) * learned.unfeatures(Tout, off.L)
    assert rel(back, e) < 1e-12
    pr = polarized.apply_P(r.ravel(), off.L, nt).reshape(-1, nt)
    assert rel(learned.unfeatures(Xin, off.L) * learned.rms(r), pr) < 1e-14
    # an all-zero network leaves the plain method unchanged
    th0 = np.zeros(learned.nparams())
    z = learned.correction(th0, r, off.L)
    assert np.count_nonzero(z) == 0
    x0, its0, _, _ = krylov.fgmres_right(A, b, K, 1e-10, 40)
    x1, its1, _, _ = krylov.fgmres_right(A, b, lambda v: K(v) + learned.correction(th0, v.reshape(-1, nt), off.L).ravel(),
                                         1e-10, 40)
    assert its0 == its1 and rel(x1, x0) < 1e-13
