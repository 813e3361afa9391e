"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no arithmetic of the method: it only draws media and
sources.  Both the CPU oracle (through the tests) and the GPU library
(through the tests and the benchmark) receive exactly these arrays.

The paper measures on Marmousi2 and BP 2004 (Section 7), which are not
available here; the media below stand in for them with the shapes, sizes and
velocity ranges of the benchmark configurations:

* ``constant``   c = 1 everywhere (homogeneous medium);
* ``grf``        smooth Gaussian random field: white N(0,1) noise on the
                 extended grid convolved (FFT, zero padded) with
                 exp(-r^2 / (2 l^2)), l = 20 grid points, min-max mapped to
                 [1.5, 4.5] (stand-in for the smoothed Marmousi2 model);
* ``layered``    piecewise-smooth layers with sinusoidal interfaces, three
                 normal faults and a high-contrast wedge, c in [1.5, 5.5]
                 (stand-in for the rough Marmousi2 / BP 2004 models).

All random draws use numpy.random.Generator(PCG64(seed)).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def constant_medium(nt: int, Nz: int, c: float = 1.0) -> np.ndarray:
    return np.full((Nz, nt), c, dtype=np.float64)


def grf_medium(nt: int, Nz: int, seed: int, corr: float = 20.0, cmin: float = 1.5, cmax: float = 4.5) -> np.ndarray:
    """Gaussian random field on the extended grid, correlation length ``corr`` grid points."""
    g = rng(seed)
    noise = g.standard_normal((Nz, nt))
    R = int(math.ceil(4 * corr))
    sz, sx = Nz + 2 * R, nt + 2 * R  # zero padding: linear, not circular, convolution
    kz = np.arange(-R, R + 1)
    ker = np.exp(-(kz[:, None] ** 2 + kz[None, :] ** 2) / (2 * corr**2))
    F = np.fft.rfft2(noise, s=(sz, sx)) * np.fft.rfft2(ker, s=(sz, sx))
    sm = np.fft.irfft2(F, s=(sz, sx))[R : R + Nz, R : R + nt]
    lo, hi = sm.min(), sm.max()
    return cmin + (cmax - cmin) * (sm - lo) / (hi - lo)


def layered_medium(nt: int, Nz: int, seed: int, n_interfaces: int = 12, cmin: float = 1.5,
                   cmax: float = 4.5, wedge_c: float = 5.5) -> np.ndarray:
    """Piecewise-smooth layered medium with faults and a wedge (grid units)."""
    g = rng(seed)
    x = np.arange(nt, dtype=np.float64)
    z = np.arange(Nz, dtype=np.float64)
    depths = np.sort(g.uniform(0.05, 0.95, n_interfaces)) * Nz
    # interfaces z_k(x) = mean depth + 3 random sinusoids, each amplitude <= 3% of depth
    surf = np.empty((n_interfaces, nt))
    for k, d in enumerate(depths):
        amp = g.uniform(0.0, 0.03, 3) * d
        wl = g.uniform(0.2, 1.0, 3) * nt
        ph = g.uniform(0, 2 * np.pi, 3)
        surf[k] = d + np.sum(amp[:, None] * np.sin(2 * np.pi * x[None, :] / wl[:, None] + ph[:, None]), axis=0)
    # three normal faults: lines at 55-75 degrees shifting depths by 2-6% of depth
    Z, X = np.meshgrid(z, x, indexing="ij")
    shift = np.zeros((Nz, nt))
    for _ in range(3):
        x0 = g.uniform(0.15, 0.85) * nt
        ang = np.deg2rad(g.uniform(55, 75))
        side = (X - x0) - (Z / np.tan(ang)) > 0
        shift += side * g.uniform(0.02, 0.06) * Z
    zz = Z - shift
    vel = np.linspace(cmin, cmax, n_interfaces + 1)
    layer_id = np.zeros((Nz, nt), dtype=np.int64)
    for k in range(n_interfaces):
        layer_id += (zz > surf[k][None, :]).astype(np.int64)
    grad = g.uniform(-0.05, 0.05, n_interfaces + 1)
    c = vel[layer_id] * (1.0 + grad[layer_id] * (X / nt - 0.5) * 2)
    # triangular high-contrast wedge
    cx, cz = g.uniform(0.3, 0.7) * nt, g.uniform(0.4, 0.7) * Nz
    w, hgt = 0.15 * nt, 0.12 * Nz
    inside = (Z <= cz) & (Z >= cz - hgt) & (np.abs(X - cx) <= w * (Z - (cz - hgt)) / hgt)
    c[inside] = wedge_c
    return np.clip(c, cmin, wedge_c)


def point_sources(nt: int, Nz: int, npml: int, h: float, positions) -> np.ndarray:
    """Discrete deltas f = 1/h^2 at physical nodes (p, q), 1-based physical indices.

    Returns (S, N_z, n_t) complex128.
    """
    pos = list(positions)
    f = np.zeros((len(pos), Nz, nt), dtype=np.complex128)
    for s, (p, q) in enumerate(pos):
        f[s, q - 1 + npml, p - 1 + npml] = 1.0 / (h * h)
    return f


def point_source_entries(npml: int, h: float, positions):
    """The nonzero entries of ``point_sources``: (rows, cols, value) with rows / cols the extended-grid
    indices of each source's node and value = 1/h^2, for building large batches in place."""
    pos = list(positions)
    rows = [q - 1 + npml for _, q in pos]
    cols = [p - 1 + npml for p, _ in pos]
    return rows, cols, 1.0 / (h * h)


def random_sources(nt: int, Nz: int, npml: int, nx: int, nz: int, seed: int, count: int) -> np.ndarray:
    """Random complex right-hand sides supported on the physical region (Section 7 times 200 random ones)."""
    g = rng(seed)
    f = np.zeros((count, Nz, nt), dtype=np.complex128)
    f[:, npml : npml + nz, npml : npml + nx] = g.standard_normal((count, nz, nx)) + 1j * g.standard_normal((count, nz, nx))
    return f


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    nx: int
    nz: int
    npml: int
    L: int
    ppw: float
    medium: str
    seed: int
    sources: tuple  # physical (p, q) pairs, 1-based
    tol: float

    @property
    def nt(self) -> int:
        return self.nx + 2 * self.npml

    @property
    def Nz(self) -> int:
        return self.nz + 2 * self.npml

    @property
    def h(self) -> float:
        return 1.0 / (self.nx + 1)

    def c_ext(self) -> np.ndarray:
        if self.medium == "constant":
            return constant_medium(self.nt, self.Nz)
        if self.medium == "grf":
            return grf_medium(self.nt, self.Nz, self.seed)
        if self.medium == "layered":
            return layered_medium(self.nt, self.Nz, self.seed)
        raise ValueError(self.medium)

    def omega(self, c_ext: np.ndarray | None = None) -> float:
        """omega at ``ppw`` points per wavelength measured at the slowest speed."""
        c = self.c_ext() if c_ext is None else c_ext
        return 2.0 * np.pi * float(c.min()) / (self.ppw * self.h)

    def f(self) -> np.ndarray:
        return point_sources(self.nt, self.Nz, self.npml, self.h, self.sources)


# 128 x 128 interior, 10-point PML, constant speed, 10 points per wavelength, L = 4,
# one unit point source at the centre, dense blocks, FP64, GMRES tolerance 1e-10.
CONSTANT_128 = Workload("constant-128x128-L4", 128, 128, 10, 4, 10.0, "constant", 0, ((64, 64),), 1e-10)
# 511 x 1023 interior, 20-point PML, Gaussian random field c in [1.5, 4.5], 10 ppw,
# L = 16, one source near the top, GMRES tolerance 1e-7.
GRF_511x1023 = Workload("grf-511x1023-L16", 511, 1023, 20, 16, 10.0, "grf", 2, ((256, 10),), 1e-7)
# 1023 x 2047 interior, 20-point PML, layered medium with faults and a wedge, L = 32,
# 256 sources on the first physical row.
LAYERED_1023x2047 = Workload("layered-1023x2047-L32", 1023, 2047, 20, 32, 10.0, "layered", 3,
                             tuple((2 + 4 * s, 1) for s in range(256)), 1e-7)

# The layered family at a quarter of the size (255 x 511, L = 8, 64 sources on the first
# physical row): the same local-problem and block shapes per layer at ~1 GB of device
# memory, for kernel captures under a profiler.
LAYERED_255x511 = Workload("layered-255x511-L8", 255, 511, 20, 8, 10.0, "layered", 3,
                           tuple((2 + 4 * s, 1) for s in range(64)), 1e-7)

WORKLOADS = {w.name: w for w in (CONSTANT_128, GRF_511x1023, LAYERED_1023x2047, LAYERED_255x511)}


def uneven_batch(count: int = 64, seed: int = 4, nmin: int = 255, nmax: int = 1023, Lmin: int = 8, Lmax: int = 32,
                 npml: int = 20, smax: int = 16, max_local_rows: int = 118) -> list:
    """An uneven batch of independent problems of the GRF family: n ~ U{nmin..nmax} odd, n_z = 2 n + 1,
    medium seed 4000 + i, ppw ~ U[8, 12] at c_min, L ~ U{Lmin..Lmax} capped so that every layer has
    npml + 2 rows and raised so that every padded local problem has at most max_local_rows rows,
    1..smax point sources in the top 10 % of the physical rows, tolerance 1e-7."""
    g = rng(seed)
    out = []
    for i in range(count):
        n = int(g.integers(nmin // 2, nmax // 2 + 1)) * 2 + 1
        n = min(max(n, nmin | 1), nmax)
        nz = 2 * n + 1
        # the near-equal split keeps the first and last interfaces outside the PML only when every
        # layer has at least npml + 2 rows
        # ... and the local problems (layer rows + 2 npml padded rows) fit the library's limit
        Nz = nz + 2 * npml
        L = min(int(g.integers(Lmin, Lmax + 1)), Nz // (npml + 2))
        L = max(L, -(-Nz // (max_local_rows - 2 * npml - 1)))
        ppw = float(g.uniform(8.0, 12.0))
        ns = int(g.integers(1, smax + 1))
        top = max(2, nz // 10)
        src = tuple((int(g.integers(1, n + 1)), int(g.integers(1, top + 1))) for _ in range(ns))
        out.append(Workload(f"grf-{n}x{nz}-L{L}-i{i}", n, nz, npml, L, ppw, "grf", 4000 + i, src, 1e-7))
    return out


def small_case(nx: int, nz: int, npml: int, L: int, ppw: float = 10.0, medium: str = "constant", seed: int = 0,
               sources=None, tol: float = 1e-10) -> Workload:
    """A reduced workload of the same structure for tests."""
    if sources is None:
        sources = ((nx // 2, nz // 2),)
    return Workload(f"{medium}-{nx}x{nz}-L{L}", nx, nz, npml, L, ppw, medium, seed, tuple(sources), tol)
