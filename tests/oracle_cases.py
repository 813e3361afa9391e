"""Small oracle fixtures shared by the oracle pin tests (CPU only)."""
import functools

import numpy as np

import workloads as W
from oracle import discretization as D
from oracle import solver as S


@functools.lru_cache(maxsize=None)
def case(nx=24, nz=30, npml=6, L=3, ppw=8.0, medium="constant", seed=0, src=None):
    wl = W.small_case(nx, nz, npml, L, ppw=ppw, medium=medium, seed=seed,
                      sources=None if src is None else (src,))
    c = wl.c_ext()
    prob = D.make_problem(c, wl.npml, wl.h, wl.omega(c))
    off = S.precompute(prob, L)
    f = wl.f()[0]
    u = S.global_solve(prob, f)
    return wl, prob, off, f, u


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))
