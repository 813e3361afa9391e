"""Learned preconditioner correction on interface traces (not in the paper).

Test infrastructure: see the package docstring.

The paper's preconditioner (Algorithm 4, two Gauss-Seidel sweeps) leaves a
defect e - K^{-1} r on any residual / error pair with M e = r.  A small
network N_theta, applied to the residual, learns that defect, and flexible
GMRES (Section 4.2, right preconditioned, which allows a preconditioner that
changes) uses z = K^{-1} v + N_theta(v).  This module is the FP64 reference of
that network: its forward pass, its loss and the exact gradient, written out
layer by layer.

Architecture (one sequence per interface and source):
  input   8 real channels over the n_t positions of an interface: Re/Im of
          the four rows of interface i of the permuted residual P r (Section
          3.5), in the order (2i, 2i+1, T+2i, T+2i+1); the output uses the
          same slots of the trace vector (u_down pair, u_up pair);
  layer 1 1D cross-correlation, 8 -> W channels, kernel K1 = 7, zero padding:
          h1[o, x] = b1[o] + sum_{c,k} W1[o, c, k] X[c, x + k - 3];
  layers 2, 3  pointwise W -> W;  layer 4  pointwise W -> 8 (no activation);
  activation GELU in its tanh form (Hendrycks & Gimpel, 2016):
          g(x) = x/2 (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3))).
The input is the residual divided by its RMS s over the whole trace vector,
and the output is multiplied by s, so the correction scales like a linear
preconditioner.  Loss: 0.5 * mean over all output entries of (y - t)^2.

Flat parameter order (the library uses the same):
  W1 (W, 8, K1) | b1 (W) | W2 (W, W) | b2 (W) | W3 (W, W) | b3 (W) | W4 (8, W) | b4 (8).
"""
from __future__ import annotations

import math

import numpy as np

CIN = 8
K1 = 7
WIDTH = 256
_C = math.sqrt(2.0 / math.pi)


def shapes(width: int = WIDTH, k1: int = K1):
    return [("W1", (width, CIN, k1)), ("b1", (width,)), ("W2", (width, width)), ("b2", (width,)),
            ("W3", (width, width)), ("b3", (width,)), ("W4", (CIN, width)), ("b4", (CIN,))]


def nparams(width: int = WIDTH, k1: int = K1) -> int:
    return sum(int(np.prod(s)) for _, s in shapes(width, k1))


def unpack(theta: np.ndarray, width: int = WIDTH, k1: int = K1) -> dict:
    out, off = {}, 0
    for name, shp in shapes(width, k1):
        n = int(np.prod(shp))
        out[name] = np.asarray(theta[off : off + n], dtype=np.float64).reshape(shp)
        off += n
    assert off == theta.size
    return out


def pack(p: dict, width: int = WIDTH, k1: int = K1) -> np.ndarray:
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel() for name, _ in shapes(width, k1)])


def gelu(x):
    return 0.5 * x * (1.0 + np.tanh(_C * (x + 0.044715 * x**3)))


def gelu_grad(x):
    u = _C * (x + 0.044715 * x**3)
    th = np.tanh(u)
    return 0.5 * (1.0 + th) + 0.5 * x * (1.0 - th**2) * _C * (1.0 + 3 * 0.044715 * x**2)


# ---- trace vectors <-> features ---------------------------------------------
def features(v: np.ndarray, L: int) -> np.ndarray:
    """(T4, n_t) complex trace vector -> (L-1, 8, n_t) real features, one row per interface."""
    T = 2 * (L - 1)
    nt = v.shape[1]
    X = np.empty((L - 1, CIN, nt))
    for i in range(L - 1):
        for q, tr in enumerate((2 * i, 2 * i + 1, T + 2 * i, T + 2 * i + 1)):
            X[i, 2 * q] = v[tr].real
            X[i, 2 * q + 1] = v[tr].imag
    return X


def unfeatures(Y: np.ndarray, L: int) -> np.ndarray:
    """Inverse of ``features``."""
    T = 2 * (L - 1)
    nt = Y.shape[2]
    v = np.zeros((2 * T, nt), dtype=np.complex128)
    for i in range(L - 1):
        for q, tr in enumerate((2 * i, 2 * i + 1, T + 2 * i, T + 2 * i + 1)):
            v[tr] = Y[i, 2 * q] + 1j * Y[i, 2 * q + 1]
    return v


# ---- the network --------------------------------------------------------------
def conv1(W1: np.ndarray, b1: np.ndarray, X: np.ndarray) -> np.ndarray:
    """Layer 1 pre-activation for X (nseq, 8, n_t): zero-padded cross-correlation over x."""
    k1 = W1.shape[2]
    half = k1 // 2
    nseq, _, nt = X.shape
    Xp = np.zeros((nseq, CIN, nt + 2 * half))
    Xp[:, :, half : half + nt] = X
    h = np.broadcast_to(b1[None, :, None], (nseq, W1.shape[0], nt)).copy()
    for k in range(k1):
        h += np.einsum("oc,scx->sox", W1[:, :, k], Xp[:, :, k : k + nt])
    return h


def forward(theta: np.ndarray, X: np.ndarray, width: int = WIDTH, k1: int = K1):
    """Network output (nseq, 8, n_t) and the intermediates the gradient needs."""
    p = unpack(theta, width, k1)
    h1 = conv1(p["W1"], p["b1"], X)
    a1 = gelu(h1)
    h2 = np.einsum("oi,six->sox", p["W2"], a1) + p["b2"][None, :, None]
    a2 = gelu(h2)
    h3 = np.einsum("oi,six->sox", p["W3"], a2) + p["b3"][None, :, None]
    a3 = gelu(h3)
    y = np.einsum("oi,six->sox", p["W4"], a3) + p["b4"][None, :, None]
    return y, (X, h1, a1, h2, a2, h3, a3)


def loss(theta: np.ndarray, X: np.ndarray, T: np.ndarray, width: int = WIDTH, k1: int = K1) -> float:
    y, _ = forward(theta, X, width, k1)
    return 0.5 * float(np.mean((y - T) ** 2))


def loss_and_grad(theta: np.ndarray, X: np.ndarray, T: np.ndarray, width: int = WIDTH, k1: int = K1):
    """Loss and its exact gradient with respect to the flat parameters (backpropagation)."""
    p = unpack(theta, width, k1)
    y, (X, h1, a1, h2, a2, h3, a3) = forward(theta, X, width, k1)
    dy = (y - T) / y.size
    g = {}
    g["W4"] = np.einsum("sox,six->oi", dy, a3)
    g["b4"] = dy.sum(axis=(0, 2))
    dh3 = np.einsum("oi,sox->six", p["W4"], dy) * gelu_grad(h3)
    g["W3"] = np.einsum("sox,six->oi", dh3, a2)
    g["b3"] = dh3.sum(axis=(0, 2))
    dh2 = np.einsum("oi,sox->six", p["W3"], dh3) * gelu_grad(h2)
    g["W2"] = np.einsum("sox,six->oi", dh2, a1)
    g["b2"] = dh2.sum(axis=(0, 2))
    dh1 = np.einsum("oi,sox->six", p["W2"], dh2) * gelu_grad(h1)
    k = p["W1"].shape[2]
    half = k // 2
    nseq, _, nt = X.shape
    Xp = np.zeros((nseq, CIN, nt + 2 * half))
    Xp[:, :, half : half + nt] = X
    g["W1"] = np.stack([np.einsum("sox,scx->oc", dh1, Xp[:, :, j : j + nt]) for j in range(k)], axis=2)
    g["b1"] = dh1.sum(axis=(0, 2))
    return 0.5 * float(np.mean((y - T) ** 2)), pack(g, width, k1)


def rms(v: np.ndarray) -> float:
    return float(np.sqrt(np.mean(np.abs(v) ** 2)))


def correction_permuted(theta: np.ndarray, pv: np.ndarray, L: int, width: int = WIDTH, k1: int = K1) -> np.ndarray:
    """N_theta applied to a permuted residual P v (T4, n_t): RMS-normalised in, rescaled out."""
    s = rms(pv)
    if s == 0.0:
        return np.zeros_like(pv)
    y, _ = forward(theta, features(pv / s, L), width, k1)
    return s * unfeatures(y, L)


def correction(theta: np.ndarray, v: np.ndarray, L: int, width: int = WIDTH, k1: int = K1) -> np.ndarray:
    """N_theta(v) for a residual v (T4, n_t) of the unpermuted jump system (the oracle's convention)."""
    from . import polarized

    nt = v.shape[1]
    return correction_permuted(theta, polarized.apply_P(v.ravel(), L, nt).reshape(-1, nt), L, width, k1)


def training_pair(split, r: np.ndarray, e: np.ndarray, L: int):
    """Features of the input P r / RMS(r) and of the target (e - K^{-1} r) / RMS(r) for a
    residual / error pair with M e = r (unpermuted jump system); K^{-1} is Algorithm 4
    with n_it = 2.  A network that reproduced the target would make K^{-1} + N_theta = M^{-1}."""
    from . import polarized

    nt = r.shape[1]
    s = rms(r)
    kr = polarized.gauss_seidel_preconditioner(split, r.ravel(), 2).reshape(-1, nt)
    pr = polarized.apply_P(r.ravel(), L, nt).reshape(-1, nt)
    return features(pr / s, L), features((e - kr) / s, L)
