"""Section 2.1 (discretization) and Section 2.2 (domain decomposition).

Test infrastructure: see the package docstring.

Conventions (the paper's, Section 2.1):
  * the extended grid has n_t = n_x + 2 n_pml columns (x) and
    N_z = n_z + 2 n_pml rows (z); arrays are indexed [row, column] and
    flattened with x fastest, as in the paper's ordering of unknowns;
  * homogeneous Dirichlet data sit one node outside the array on every side;
  * H = -d_xx - d_zz - m omega^2 with d_x -> alpha_x d_x,
    alpha = 1 / (1 + i sigma / omega), sigma quadratic in the depth d into
    the PML, sigma = (C / delta) (d / delta)^2, delta = n_pml h.

Reading (the paper leaves where sigma starts implicit): the PML edge of a line
of n unknowns is at index n_pml - 1 on the left and n - n_pml on the right,
sigma = 0 between them (half-indices included) and the depth is measured from
that edge in units of h.  The Dirichlet node (index -1 or n) is then exactly
delta away from the edge.  The same rule, applied to a local problem whose
rows are padded with n_pml PML rows beyond an internal interface, makes
alpha_z = 1 on the local rows 0, 1/2, n+1/2, n+1 that the incomplete Green's
integrals of Definition 2 rely on (Appendix A derives them by summation by
parts with unit coefficients there).
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.sparse as sp


def default_pml_strength(c_max: float) -> float:
    """PML strength C, a tuning parameter in Section 2.1.

    Reading: choose C so that the continuous round trip through the layer
    damps a wave of speed c_max by 1e-6; the integral of sigma over the layer
    is C/3, so exp(-2 C / (3 c_max)) = 1e-6.
    """
    return 1.5 * c_max * np.log(1.0e6)


def pml_alpha(pos: np.ndarray, n: int, npml: int, h: float, omega: float, C: float) -> np.ndarray:
    """alpha(pos) = 1 / (1 + i sigma(pos) / omega) on a line of n unknowns (Section 2.1).

    pos may hold integer (node) or half-integer (midpoint) indices.
    """
    pos = np.asarray(pos, dtype=np.float64)
    depth = np.maximum(np.maximum((npml - 1) - pos, pos - (n - npml)), 0.0) * h
    delta = npml * h
    sigma = (C / delta) * (depth / delta) ** 2
    return 1.0 / (1.0 + 1j * sigma / omega)


def helmholtz_operator(m: np.ndarray, npml: int, h: float, omega: float, C: float) -> sp.csr_matrix:
    """Sparse 5-point Helmholtz operator with PML on a grid m[rows, cols] (Section 2.1).

    (H u)_{p,q} = - a_x(p) [a_x(p+1/2)(u_{p+1}-u_p) - a_x(p-1/2)(u_p-u_{p-1})] / h^2
                  - a_z(q) [a_z(q+1/2)(u_{q+1}-u_q) - a_z(q-1/2)(u_q-u_{q-1})] / h^2
                  - omega^2 m_{p,q} u_{p,q}
    with zero Dirichlet data outside the array.  Unknowns are ordered with x
    (columns) fastest.  Away from the PML this is the plain 5-point stencil
    of the paper's interior equation.
    """
    nrow, ncol = m.shape
    p = np.arange(ncol)
    q = np.arange(nrow)
    ax, axp, axm = (pml_alpha(p + s, ncol, npml, h, omega, C) for s in (0.0, 0.5, -0.5))
    az, azp, azm = (pml_alpha(q + s, nrow, npml, h, omega, C) for s in (0.0, 0.5, -0.5))
    inv_h2 = 1.0 / (h * h)

    idx = np.arange(nrow * ncol).reshape(nrow, ncol)
    rows, cols, vals = [], [], []

    def add(r, c, v):
        rows.append(r.ravel())
        cols.append(c.ravel())
        vals.append(np.broadcast_to(v, r.shape).ravel())

    center = (ax * (axp + axm))[None, :] * inv_h2 + (az * (azp + azm))[:, None] * inv_h2 - omega**2 * m
    add(idx, idx, center)
    # west / east neighbours (x direction)
    add(idx[:, 1:], idx[:, :-1], np.broadcast_to(-(ax * axm)[None, 1:] * inv_h2, (nrow, ncol - 1)))
    add(idx[:, :-1], idx[:, 1:], np.broadcast_to(-(ax * axp)[None, :-1] * inv_h2, (nrow, ncol - 1)))
    # north / south neighbours (z direction)
    add(idx[1:, :], idx[:-1, :], np.broadcast_to(-(az * azm)[1:, None] * inv_h2, (nrow - 1, ncol)))
    add(idx[:-1, :], idx[1:, :], np.broadcast_to(-(az * azp)[:-1, None] * inv_h2, (nrow - 1, ncol)))

    N = nrow * ncol
    H = sp.coo_matrix(
        (np.concatenate(vals).astype(np.complex128), (np.concatenate(rows), np.concatenate(cols))),
        shape=(N, N),
    )
    return H.tocsr()


@dataclasses.dataclass(frozen=True)
class Problem:
    """The data of Section 2.1: squared slowness on the extended grid, h, omega, PML."""

    c_ext: np.ndarray  # (N_z, n_t) wave speed on the extended grid, x fastest
    npml: int
    h: float
    omega: float
    C: float

    @property
    def m(self) -> np.ndarray:
        return 1.0 / self.c_ext**2

    @property
    def nt(self) -> int:
        return self.c_ext.shape[1]

    @property
    def Nz(self) -> int:
        return self.c_ext.shape[0]


def make_problem(c_ext: np.ndarray, npml: int, h: float, omega: float, C: float | None = None) -> Problem:
    c_ext = np.ascontiguousarray(c_ext, dtype=np.float64)
    if C is None:
        C = default_pml_strength(float(c_ext.max()))
    return Problem(c_ext=c_ext, npml=npml, h=h, omega=omega, C=C)


def global_operator(prob: Problem) -> sp.csr_matrix:
    """The global matrix H of the discrete Helmholtz equation (Section 2.1)."""
    return helmholtz_operator(prob.m, prob.npml, prob.h, prob.omega, prob.C)


# ----------------------------------------------------------------------------
# Section 2.2: layered decomposition
# ----------------------------------------------------------------------------


def layer_partition(Nz: int, L: int) -> np.ndarray:
    """Cumulative row offsets n_c (length L+1) of a near-equal split of N_z rows.

    The paper only asks for an increasing sequence n_c^l (Section 2.2).
    Reading: the first (N_z mod L) layers get one extra row.  Offsets are
    0-based array rows, so layer l covers rows n_c[l] .. n_c[l+1]-1.
    """
    base, extra = divmod(Nz, L)
    sizes = np.full(L, base, dtype=np.int64)
    sizes[:extra] += 1
    return np.concatenate([[0], np.cumsum(sizes)])


def check_partition(Nz: int, npml: int, nc: np.ndarray) -> None:
    """Every interface must sit where the global PML vanishes (Section 2.2).

    The traces at rows n, n+1 of a layer and their half-rows must be outside
    the global PML, which holds when npml + 1 <= n_c^l <= N_z - npml - 1 for
    every internal interface; every layer needs n^l >= 3 rows.
    """
    sizes = np.diff(nc)
    if np.any(sizes < 3):
        raise ValueError("every layer needs at least 3 rows")
    for s in nc[1:-1]:
        if not (npml + 1 <= s <= Nz - npml - 1):
            raise ValueError(f"interface at row {s} lies in or next to the PML")


@dataclasses.dataclass(frozen=True)
class Layer:
    """Local problem of layer l (Section 2.2) with its index bookkeeping.

    Local rows run over the layer's own rows 1..n (paper numbering) plus
    n_pml padded PML rows beyond every internal interface; the first and last
    layers keep the global PML on their outer side and get no padding there.
    ``pad_top`` is the number of padded rows above paper row 1, so paper row j
    is local array row j - 1 + pad_top.
    """

    index: int
    start: int  # first global array row of the layer
    n: int  # rows of the layer (n^l)
    pad_top: int
    pad_bot: int
    m_local: np.ndarray  # (nloc, n_t) normally extended squared slowness

    @property
    def nloc(self) -> int:
        return self.pad_top + self.n + self.pad_bot

    def row(self, j: int) -> int:
        """Local array row of the paper's local row index j (q = n_c^l + j)."""
        return j - 1 + self.pad_top


def make_layer(prob: Problem, nc: np.ndarray, l: int) -> Layer:
    """Extended local model (the normal extension m~ of Section 2.2)."""
    L = len(nc) - 1
    start, stop = int(nc[l]), int(nc[l + 1])
    n = stop - start
    pad_top = prob.npml if l > 0 else 0
    pad_bot = prob.npml if l < L - 1 else 0
    m = prob.m
    rows = [m[start : start + 1]] * pad_top + [m[start:stop]] + [m[stop - 1 : stop]] * pad_bot
    m_local = np.ascontiguousarray(np.concatenate(rows, axis=0))
    return Layer(index=l, start=start, n=n, pad_top=pad_top, pad_bot=pad_bot, m_local=m_local)


def local_operator(prob: Problem, layer: Layer) -> sp.csr_matrix:
    """H^l: the local problem of Section 2.2 on the padded grid of layer l."""
    return helmholtz_operator(layer.m_local, prob.npml, prob.h, prob.omega, prob.C)


def physical_mask(prob: Problem, nx: int, nz: int) -> np.ndarray:
    """Boolean mask of the physical region Omega (PML excluded) on the extended grid."""
    mask = np.zeros((prob.Nz, prob.nt), dtype=bool)
    mask[prob.npml : prob.npml + nz, prob.npml : prob.npml + nx] = True
    return mask
