"""The precision choices of the mixed form, checked on the oracle (CPU only).

FP16 preconditioner blocks: each block row scaled by a power of two into [2^13, 2^14) of its
largest |Re|, |Im| and rounded to FP16.  Flexible GMRES with the Gauss-Seidel preconditioner
(Algorithm 4) built on those blocks, applied to the exact polarized system, must still reach
the tolerance, with at most one more iteration than with the exact preconditioner.

Relaxed matvecs (inexact Krylov): once the least-squares residual estimate is below
1e4 tol ||b||, the matvec may use complex64 blocks and a complex64 input; the flexible GMRES
cycle must end with the same iteration count (up to one) and a true residual below tol.
"""
import numpy as np

from oracle import krylov, polarized
from oracle import solver as S
from oracle.integral import BlockSystem

from .oracle_cases import case


def _rounded_system(system, fn):
    out = BlockSystem(system.nrows, system.ncols, system.nt)
    for r, terms in enumerate(system.rows):
        out.add(r, [(c, blk if np.isscalar(blk) else fn(blk)) for c, blk in terms])
    return out


def _fp16_rows(blk):
    m = np.maximum(np.abs(blk.real), np.abs(blk.imag)).max(axis=1)
    ex = np.frexp(np.where(m > 0, m, 1.0))[1]
    p = np.where(m > 0, 14 - ex, 0).astype(float)[:, None]
    re = (blk.real * 2.0 ** p).astype(np.float16).astype(np.float64)
    im = (blk.imag * 2.0 ** p).astype(np.float16).astype(np.float64)
    return (re + 1j * im) * 2.0 ** (-p)


def _c64(blk):
    return blk.astype(np.complex64).astype(np.complex128)


def _setup():
    wl, prob, off, f, u = case(nx=40, nz=60, npml=8, L=4, ppw=8.0, medium="grf", seed=11)
    b = S.polarized_rhs(off, f)
    return off, b


def test_fp16_preconditioner_blocks_cost_at_most_one_iteration():
    off, b = _setup()
    A = off.system.apply
    tol = 1e-8
    exact = lambda v: polarized.gauss_seidel_preconditioner(off.split, v, 2)  # noqa: E731
    split16 = polarized.Splitting(_rounded_system(off.system, _fp16_rows), off.L)
    half = lambda v: polarized.gauss_seidel_preconditioner(split16, v, 2)  # noqa: E731
    v = np.random.default_rng(3).standard_normal(b.size) + 0j
    z0, z1 = exact(v), half(v)
    assert 1e-6 < np.linalg.norm(z1 - z0) / np.linalg.norm(z0) < 1e-2  # FP16 accuracy, not exact
    _, its0, rel0, _ = krylov.fgmres_right(A, b, exact, tol, 60)
    _, its1, rel1, _ = krylov.fgmres_right(A, b, half, tol, 60)
    assert rel0 <= tol and rel1 <= tol
    assert its1 <= its0 + 1


def _relaxed_fgmres(A, A32, b, Minv, tol, max_it, relax):
    """One flexible-GMRES cycle (modified Gram-Schmidt, least squares by lstsq) whose matvec is A32 once the
    residual estimate is below relax * tol * ||b||; returns x, iterations, relaxed matvecs."""
    beta = np.linalg.norm(b)
    V = [b / beta]
    Z, H = [], np.zeros((max_it + 1, max_it), dtype=complex)
    est, relaxed = beta, 0
    for j in range(max_it):
        z = Minv(V[j])
        Z.append(z)
        use32 = j > 0 and est <= relax * tol * beta
        relaxed += int(use32)
        w = A32(z) if use32 else A(z)
        for i in range(j + 1):
            H[i, j] = np.vdot(V[i], w)
            w = w - H[i, j] * V[i]
        H[j + 1, j] = np.linalg.norm(w)
        V.append(w / H[j + 1, j])
        e1 = np.zeros(j + 2, dtype=complex)
        e1[0] = beta
        y = np.linalg.lstsq(H[: j + 2, : j + 1], e1, rcond=None)[0]
        est = np.linalg.norm(e1 - H[: j + 2, : j + 1] @ y)
        if est <= tol * beta:
            break
    x = sum(yi * zi for yi, zi in zip(y, Z))
    return x, j + 1, relaxed


def test_relaxed_complex64_matvecs_keep_the_tolerance():
    off, b = _setup()
    A = off.system.apply
    sys32 = _rounded_system(off.system, _c64)
    A32 = lambda x: sys32.apply(x.astype(np.complex64).astype(np.complex128))  # noqa: E731
    Minv = lambda v: polarized.gauss_seidel_preconditioner(off.split, v, 2)  # noqa: E731
    for tol in (1e-7, 1e-10):
        x0, its0, n0 = _relaxed_fgmres(A, A32, b, Minv, tol, 60, relax=0.0)
        x1, its1, n1 = _relaxed_fgmres(A, A32, b, Minv, tol, 60, relax=1e4)
        assert n0 == 0 and n1 >= 1
        assert abs(its1 - its0) <= 1
        true = np.linalg.norm(b - A(x1)) / np.linalg.norm(b)
        assert true <= tol, (tol, true)
