"""The chunked local-solve scheme (an exact reorganisation of the block substitutions of
the local factorization, Section 2.2 / Algorithm 1), checked in numpy on a local problem of
the oracle, CPU only.

The layer's operator H^l, reordered column-major (z fastest), is block tridiagonal in x with
diagonal couplings W_i, E_i.  Forward y_i = S_i^{-1}(f_i - W_i y_{i-1}) and backward
x_i = y_i - S_i^{-1} E_i x_{i+1} are cut into chunks; the chunks are solved from zero
boundary values, the boundary values follow from the transfer matrices
Phi_k = A_{b_k}...A_{a_k}, M_k = sum_j (B_{a_k}...B_{j-1}) Phi_j, Psi_k = B_{a_k}...B_{b_k}
(A_i = -S_i^{-1} diag(W_i), B_i = -S_i^{-1} diag(E_i)), formed by the forward accumulation
the library uses (Phi <- A_j Phi, M <- M + G Phi, G <- G B_j), and the chunks are solved
again.  The result must equal the sparse direct solve of H^l to rounding, for any chunking.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import workloads as W
from oracle import discretization as D


def _blocks(n_x=60, n_z=48, npml=8, L=3, layer=1):
    wl = W.small_case(n_x, n_z, npml, L, medium="grf", seed=4)
    c = wl.c_ext()
    prob = D.make_problem(c, wl.npml, wl.h, wl.omega(c))
    nc = D.layer_partition(prob.Nz, L)
    lay = D.make_layer(prob, nc, layer)
    H = D.local_operator(prob, lay).tocsr()
    n, nt = lay.nloc, prob.nt
    perm = np.array([z * nt + x for x in range(nt) for z in range(n)])  # x-major: index x * n + z
    Hp = H[perm][:, perm].tocsr()
    Dd, Wd, Ed = [], [], []
    for i in range(nt):
        rows = Hp[i * n:(i + 1) * n, :]
        Dd.append(rows[:, i * n:(i + 1) * n].toarray())
        Wd.append(np.diag(rows[:, (i - 1) * n:i * n].toarray()) if i > 0 else np.zeros(n))
        Ed.append(np.diag(rows[:, (i + 1) * n:(i + 2) * n].toarray()) if i < nt - 1 else np.zeros(n))
    return Hp, Dd, Wd, Ed, n, nt


def _chunked_solve(Sinv, Wd, Ed, f, K):
    nt, n = f.shape
    a = [k * nt // K for k in range(K)]
    b = [(k + 1) * nt // K - 1 for k in range(K)]

    def chunk(k, beta, gamma):
        y, prev = {}, beta
        for i in range(a[k], b[k] + 1):
            y[i] = Sinv[i] @ (f[i] - Wd[i] * prev)
            prev = y[i]
        x, nxt = {}, gamma
        for i in range(b[k], a[k] - 1, -1):
            x[i] = y[i] - Sinv[i] @ (Ed[i] * nxt)
            nxt = x[i]
        return y, x

    Phi_k, M_k, Psi_k = [], [], []
    for k in range(K):
        Phi = np.eye(n, dtype=complex)
        G = np.eye(n, dtype=complex)
        M = np.zeros((n, n), complex)
        for j in range(a[k], b[k] + 1):
            Phi = -Sinv[j] @ (Wd[j][:, None] * Phi)
            M = M + G @ Phi
            G = -(G @ Sinv[j]) * Ed[j][None, :]
        Phi_k.append(Phi)
        M_k.append(M)
        Psi_k.append(G)
    z = np.zeros(n, complex)
    yb, xa = [], []
    for k in range(K):
        y, x = chunk(k, z, z)
        yb.append(y[b[k]])
        xa.append(x[a[k]])
    beta, gamma = [z] * K, [z] * K
    for k in range(K - 1):
        beta[k + 1] = yb[k] + Phi_k[k] @ beta[k]
    for k in range(K - 1, 0, -1):
        gamma[k - 1] = xa[k] + M_k[k] @ beta[k] + Psi_k[k] @ gamma[k]
    out = np.zeros((nt, n), complex)
    for k in range(K):
        _, x = chunk(k, beta[k], gamma[k])
        for i in range(a[k], b[k] + 1):
            out[i] = x[i]
    return out


@pytest.mark.parametrize("K", [1, 2, 5, 11])
def test_chunked_substitutions_equal_the_direct_solve(K):
    Hp, Dd, Wd, Ed, n, nt = _blocks()
    Sinv = []
    for i in range(nt):
        S = Dd[i] - (Wd[i][:, None] * Sinv[i - 1] * Ed[i - 1][None, :] if i > 0 else 0)
        Sinv.append(np.linalg.inv(S))
    g = np.random.default_rng(K)
    f = g.standard_normal((nt, n)) + 1j * g.standard_normal((nt, n))
    ref = spla.spsolve(Hp.tocsc(), f.ravel()).reshape(nt, n)
    got = _chunked_solve(Sinv, Wd, Ed, f, K)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-12


def test_point_source_in_the_last_chunk_matches_the_direct_solve():
    Hp, Dd, Wd, Ed, n, nt = _blocks()
    Sinv = []
    for i in range(nt):
        S = Dd[i] - (Wd[i][:, None] * Sinv[i - 1] * Ed[i - 1][None, :] if i > 0 else 0)
        Sinv.append(np.linalg.inv(S))
    f = np.zeros((nt, n), complex)
    f[nt - 5, n // 2] = 1.0  # a source in the last chunk: every earlier chunk is reached only through gamma
    ref = spla.spsolve(Hp.tocsc(), f.ravel()).reshape(nt, n)
    got = _chunked_solve(Sinv, Wd, Ed, f, 6)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-12
    assert np.abs(got[0]).max() > 0  # the field reaches the first column
