"""GB300 (sm_103a) implementation of the method of polarized traces for the 2D Helmholtz equation.

Python face of the C library ``libpolartrace`` (``include/polartrace.h``).
PyTorch only provides device memory and the stream; every step of the method
(offline factorisation and Green's-matrix extraction, the interface
right-hand side, flexible GMRES with the Gauss-Seidel sweep preconditioner,
the volume reconstruction) runs in the library's CUDA kernels.

    solver = PolarTrace(nx, nz, npml, L, h, omega, c_ext_cuda)
    u, traces, iters, relres = solver.solve(f_cuda, tol=1e-7)
"""
from __future__ import annotations

import ctypes as C
import math

import torch

from ._lib import PT_FP64, PT_MIXED_FP32, PT_MIXED_TC, PT_OPT_LAYER_GROUP, PT_OPT_LEARNED, PT_OPT_LOCAL_SOLVE, PT_OPT_PRECOND_FP16, PT_OPT_RELAX, PT_OPT_RESTART, PT_OPT_SWEEP, Params, PolarTraceError, check, lib

__all__ = ["PolarTrace", "PolarTraceError", "solve_many", "PT_FP64", "PT_MIXED_FP32", "PT_MIXED_TC", "PT_OPT_LAYER_GROUP", "PT_OPT_LEARNED", "PT_OPT_LOCAL_SOLVE", "PT_OPT_PRECOND_FP16", "PT_OPT_RELAX", "PT_OPT_RESTART", "PT_OPT_SWEEP", "default_pml_strength",
           "layer_partition"]


def default_pml_strength(c_max: float) -> float:
    """C such that the continuous round trip through the PML damps speed c_max by 1e-6 (C = 1.5 c_max ln 1e6)."""
    return 1.5 * c_max * math.log(1.0e6)


def _params(nx, nz, npml, L, h, omega, pml_C, precision, gs_iters, max_sources, max_krylov, plr=0, plr_eps=1e-9,
            plr_rmax=24, learned=0, layer_rows=None):
    """(pt_params, keep-alive) - the int32 array behind layer_rows must outlive the call that reads it."""
    rows = None
    if layer_rows is not None:
        rows = (C.c_int32 * len(layer_rows))(*[int(v) for v in layer_rows])
    p = Params(nx, nz, npml, L, h, omega, pml_C, precision, gs_iters, max_sources, max_krylov, plr, plr_eps,
               plr_rmax, learned, C.cast(rows, C.POINTER(C.c_int32)) if rows is not None else None)
    return p, rows


def layer_partition(nx, nz, npml, L, layer_rows=None) -> list:
    """Row offsets of the library's layer split (Section 2.2), or of the given rows per layer."""
    p, _keep = _params(nx, nz, npml, L, 1.0, 1.0, 1.0, PT_FP64, 2, 1, 1, layer_rows=layer_rows)
    out = (C.c_int32 * (L + 1))()
    check(lib().pt_layer_partition(C.byref(p), out), "pt_layer_partition")
    return list(out)


def _ptr(t: torch.Tensor) -> int:
    return t.data_ptr()


def solve_many(solvers, fs, tol: float = 1e-7, max_it: int | None = None, want_u: bool = True):
    """Uneven batch: solve every solver's sources concurrently (pt_solve_many).  Give each solver its own
    stream (PolarTrace(..., stream=torch.cuda.Stream())) for the solves to overlap.  Returns
    (u list, iterations list, true relative residual list)."""
    n = len(solvers)
    if n != len(fs):
        raise ValueError("one source tensor per solver")
    us = []
    for sv, f in zip(solvers, fs):
        sv._check_src(f)
        us.append(torch.empty_like(f) if want_u else None)
    if max_it is None:
        max_it = min(sv.max_krylov for sv in solvers)
    vp = C.c_void_p
    ctxs = (vp * n)(*[sv._ctx.value for sv in solvers])
    nsrc = (C.c_int32 * n)(*[f.shape[0] for f in fs])
    fp = (vp * n)(*[f.data_ptr() for f in fs])
    up = (vp * n)(*[u.data_ptr() for u in us]) if want_u else None
    scr = (vp * n)(*[sv._scratch.data_ptr() for sv in solvers])
    scb = (C.c_size_t * n)(*[sv._scratch.numel() for sv in solvers])
    tot = sum(f.shape[0] for f in fs)
    iters = (C.c_int32 * tot)()
    rel = (C.c_double * tot)()
    status = (C.c_int32 * n)()
    torch.cuda.synchronize()
    check(lib().pt_solve_many(n, ctxs, nsrc, fp, up, tol, max_it, scr, scb, iters, rel, status), "pt_solve_many")
    torch.cuda.synchronize()
    out_i, out_r, o = [], [], 0
    for f in fs:
        out_i.append(list(iters[o:o + f.shape[0]]))
        out_r.append(list(rel[o:o + f.shape[0]]))
        o += f.shape[0]
    return us, out_i, out_r


class PolarTrace:
    """An offline-prepared solver (Algorithm 1 on the GPU) for one medium and frequency."""

    def __init__(self, nx: int, nz: int, npml: int, L: int, h: float, omega: float, c_ext: torch.Tensor,
                 pml_C: float | None = None, precision: int = PT_FP64, gs_iters: int = 2, max_sources: int = 1,
                 max_krylov: int = 40, stream: torch.cuda.Stream | None = None, plr: bool = False,
                 plr_eps: float = 1e-9, plr_rmax: int = 24, learned: bool = False, layer_rows=None):
        if not (c_ext.is_cuda and c_ext.dtype == torch.float64 and c_ext.is_contiguous()):
            raise ValueError("c_ext must be a contiguous float64 CUDA tensor of shape (N_z, n_t)")
        self.nx, self.nz, self.npml, self.L = nx, nz, npml, L
        self.nt, self.Nz = nx + 2 * npml, nz + 2 * npml
        if tuple(c_ext.shape) != (self.Nz, self.nt):
            raise ValueError(f"c_ext must have shape {(self.Nz, self.nt)}")
        if pml_C is None:
            pml_C = default_pml_strength(float(c_ext.max()))
        self.params, self._rows = _params(nx, nz, npml, L, h, omega, pml_C, precision, gs_iters, max_sources,
                                          max_krylov, int(plr), plr_eps, plr_rmax, int(learned), layer_rows)
        self.max_sources, self.max_krylov = max_sources, max_krylov
        self.device = c_ext.device
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        L_ = lib()
        pb, sb, vb = C.c_size_t(), C.c_size_t(), C.c_size_t()
        check(L_.pt_workspace_size(C.byref(self.params), C.byref(pb), C.byref(sb), C.byref(vb)), "pt_workspace_size")
        self.persistent_bytes, self.setup_bytes, self.solve_bytes = pb.value, sb.value, vb.value
        self._persistent = torch.empty(pb.value, dtype=torch.uint8, device=self.device)
        setup = torch.empty(max(sb.value, 256), dtype=torch.uint8, device=self.device)
        self._scratch = torch.empty(max(vb.value, 256), dtype=torch.uint8, device=self.device)
        ctx = C.c_void_p()
        with torch.cuda.stream(self.stream):
            check(L_.pt_create(C.byref(self.params), _ptr(c_ext), _ptr(self._persistent), pb.value, _ptr(setup),
                               sb.value, C.c_void_p(self.stream.cuda_stream), C.byref(ctx)), "pt_create")
        del setup
        self._ctx = ctx
        self.T4 = 4 * (L - 1)

    def __del__(self):
        ctx = getattr(self, "_ctx", None)
        if ctx:
            lib().pt_destroy(ctx)
            self._ctx = None

    # ---- online -----------------------------------------------------------
    def _check_src(self, f: torch.Tensor) -> int:
        if f.dim() == 2:
            f = f.unsqueeze(0)
        if not (f.is_cuda and f.dtype == torch.complex128 and f.is_contiguous()):
            raise ValueError("f must be a contiguous complex128 CUDA tensor (S, N_z, n_t)")
        if tuple(f.shape[1:]) != (self.Nz, self.nt):
            raise ValueError(f"f must have shape (S, {self.Nz}, {self.nt})")
        return f.shape[0]

    def solve(self, f: torch.Tensor, tol: float = 1e-7, max_it: int | None = None, want_u: bool = True,
              want_traces: bool = True, u: torch.Tensor | None = None, allow_not_converged: bool = False):
        """Algorithm 2 for S sources.  Returns (u, traces, iterations, true relative residuals)."""
        squeeze = f.dim() == 2
        if squeeze:
            f = f.unsqueeze(0)
        S = self._check_src(f)
        if max_it is None:
            max_it = self.max_krylov
        if want_u and u is None:
            u = torch.empty_like(f)
        tr = torch.empty((S, self.T4, self.nt), dtype=torch.complex128, device=self.device) if want_traces else None
        iters = (C.c_int32 * S)()
        rel = (C.c_double * S)()
        st = lib().pt_solve(self._ctx, S, _ptr(f), _ptr(u) if want_u else None, _ptr(tr) if want_traces else None,
                            tol, max_it, _ptr(self._scratch), self._scratch.numel(), iters, rel)
        check(st, "pt_solve", allow=(5,) if allow_not_converged else ())
        out_u = u if want_u else None
        if squeeze:
            out_u = out_u[0] if out_u is not None else None
            tr = tr[0] if tr is not None else None
        return out_u, tr, list(iters), list(rel)

    def solve_gs(self, f: torch.Tensor, tol: float = 1e-7, max_it: int = 200, want_u: bool = True,
                 want_traces: bool = True, allow_not_converged: bool = False):
        """Algorithm 3 (Gauss-Seidel iteration as the solver) for S sources.  Returns (u, traces, iterations,
        FP64 true relative residuals of the polarized system)."""
        squeeze = f.dim() == 2
        if squeeze:
            f = f.unsqueeze(0)
        S = self._check_src(f)
        u = torch.empty_like(f) if want_u else None
        tr = torch.empty((S, self.T4, self.nt), dtype=torch.complex128, device=self.device) if want_traces else None
        iters = (C.c_int32 * S)()
        rel = (C.c_double * S)()
        st = lib().pt_solve_gs(self._ctx, S, _ptr(f), _ptr(u) if want_u else None, _ptr(tr) if want_traces else None,
                               tol, max_it, _ptr(self._scratch), self._scratch.numel(), iters, rel)
        check(st, "pt_solve_gs", allow=(5,) if allow_not_converged else ())
        if squeeze:
            u = u[0] if u is not None else None
            tr = tr[0] if tr is not None else None
        return u, tr, list(iters), list(rel)

    def host_scratch_bytes(self) -> int:
        return self.solve_bytes + 2 * self.max_sources * self.Nz * self.nt * 16 + 4096

    def solve_host(self, f_host: torch.Tensor, u_host: torch.Tensor, tol: float = 1e-7, max_it: int | None = None,
                   scratch: torch.Tensor | None = None):
        """Algorithm 2 through pt_solve_host: f and u in host memory (pinned for full copy speed)."""
        if f_host.is_cuda or u_host.is_cuda:
            raise ValueError("solve_host takes host tensors")
        S = f_host.shape[0]
        if scratch is None:
            scratch = torch.empty(self.host_scratch_bytes(), dtype=torch.uint8, device=self.device)
        iters = (C.c_int32 * S)()
        rel = (C.c_double * S)()
        check(lib().pt_solve_host(self._ctx, S, _ptr(f_host), _ptr(u_host), tol, max_it or self.max_krylov,
                                  _ptr(scratch), scratch.numel(), iters, rel), "pt_solve_host")
        return list(iters), list(rel)

    def last_solve_stats(self):
        n = C.c_int64()
        m = C.c_int32()
        check(lib().pt_last_solve_stats(self._ctx, C.byref(n), C.byref(m)), "pt_last_solve_stats")
        return n.value, m.value

    def last_solve_cycles(self):
        """(restart cycles, cycles that applied the learned correction) of the last solve."""
        a, b = C.c_int32(), C.c_int32()
        check(lib().pt_last_solve_cycles(self._ctx, C.byref(a), C.byref(b)), "pt_last_solve_cycles")
        return a.value, b.value

    def last_solve_relaxed(self) -> int:
        """Matvecs of the last solve that ran in FP32 under PT_OPT_RELAX."""
        a = C.c_int32()
        check(lib().pt_last_solve_relaxed(self._ctx, C.byref(a)), "pt_last_solve_relaxed")
        return a.value

    # ---- building blocks (testing) -----------------------------------------
    def _vec(self, S):
        return torch.empty((S, self.T4, self.nt), dtype=torch.complex128, device=self.device)

    def apply(self, which: str, x: torch.Tensor, working: bool = True) -> torch.Tensor:
        """One operator ('matvec', 'R', 'Dinv') in the solver's working representation (or dense FP64);
        'restart': P M in the arithmetic of the explicit residual between restart cycles."""
        y = torch.empty_like(x)
        w = {"matvec": 0, "R": 1, "Dinv": 2, "restart": 3}[which]
        check(lib().pt_apply(self._ctx, w, int(working), x.shape[0], _ptr(x), _ptr(y), _ptr(self._scratch),
                             self._scratch.numel()), "pt_apply")
        return y

    def volume_residual(self, f: torch.Tensor, u: torch.Tensor) -> list:
        """FP64 ||f - H u|| / ||f|| per source on the extended grid (Section 2.1)."""
        if f.dim() == 2:
            f, u = f.unsqueeze(0), u.unsqueeze(0)
        S = f.shape[0]
        out = (C.c_double * S)()
        check(lib().pt_volume_residual(self._ctx, S, _ptr(f), _ptr(u), out, _ptr(self._scratch),
                                       self._scratch.numel()), "pt_volume_residual")
        return list(out)

    # ---- learned correction of the preconditioner ------------------------------
    @staticmethod
    def correction_nparams() -> int:
        n = C.c_int64()
        check(lib().pt_correction_nparams(C.byref(n)), "pt_correction_nparams")
        return n.value

    def set_correction(self, theta) -> None:
        """Network weights (flat float32, the order of include/polartrace.h) from host memory."""
        t = torch.as_tensor(theta, dtype=torch.float32).contiguous().cpu()
        check(lib().pt_set_correction(self._ctx, t.data_ptr(), t.numel()), "pt_set_correction")

    def get_correction(self) -> torch.Tensor:
        t = torch.empty(self.correction_nparams(), dtype=torch.float32)
        check(lib().pt_get_correction(self._ctx, t.data_ptr(), t.numel()), "pt_get_correction")
        return t

    def _nn_scratch(self, nseq: int) -> torch.Tensor:
        b = C.c_size_t()
        check(lib().pt_correction_scratch_bytes(self._ctx, nseq, C.byref(b)), "pt_correction_scratch_bytes")
        return torch.empty(max(b.value, 256), dtype=torch.uint8, device=self.device)

    def correction_forward(self, x: torch.Tensor) -> torch.Tensor:
        """N_theta on raw features x (8, nseq * n_t) float32 CUDA."""
        nseq = x.shape[1] // self.nt
        y = torch.empty_like(x)
        sc = self._nn_scratch(nseq)
        check(lib().pt_correction_forward(self._ctx, nseq, _ptr(x), _ptr(y), _ptr(sc), sc.numel()),
              "pt_correction_forward")
        return y

    def correction_grad(self, x: torch.Tensor, t: torch.Tensor):
        """(loss, gradient) of 0.5 mean (N_theta(x) - t)^2 at the BF16 weights."""
        nseq = x.shape[1] // self.nt
        g = torch.empty(self.correction_nparams(), dtype=torch.float32, device=self.device)
        sc = self._nn_scratch(nseq)
        loss = C.c_double()
        check(lib().pt_correction_grad(self._ctx, nseq, _ptr(x), _ptr(t), C.byref(loss), _ptr(g), _ptr(sc),
                                       sc.numel()), "pt_correction_grad")
        return loss.value, g

    def train_correction(self, r: torch.Tensor, e: torch.Tensor, steps: int, batch: int, lr: float = 1e-3,
                         seed: int = 0):
        """Adam on (residual, error) pairs; returns (first, last) minibatch loss."""
        n = r.shape[0]
        b = C.c_size_t()
        check(lib().pt_train_bytes(self._ctx, n, batch, C.byref(b)), "pt_train_bytes")
        sc = torch.empty(max(b.value, 256), dtype=torch.uint8, device=self.device)
        l0, l1 = C.c_double(), C.c_double()
        check(lib().pt_train_correction(self._ctx, n, _ptr(r), _ptr(e), steps, batch, lr, seed, C.byref(l0),
                                        C.byref(l1), _ptr(sc), sc.numel()), "pt_train_correction")
        return l0.value, l1.value

    def apply_correction(self, v: torch.Tensor) -> torch.Tensor:
        z = torch.empty_like(v)
        check(lib().pt_apply_correction(self._ctx, v.shape[0], _ptr(v), _ptr(z), _ptr(self._scratch),
                                        self._scratch.numel()), "pt_apply_correction")
        return z

    def set_option(self, option: int, value: int) -> None:
        """Tuning option (PT_OPT_LAYER_GROUP: sources per CTA of the batched local solves)."""
        check(lib().pt_set_option(self._ctx, int(option), int(value)), "pt_set_option")

    def plr_stats(self):
        n = C.c_int64()
        m = C.c_int32()
        check(lib().pt_plr_stats(self._ctx, C.byref(n), C.byref(m)), "pt_plr_stats")
        return n.value, m.value

    def matvec(self, x: torch.Tensor) -> torch.Tensor:
        y = torch.empty_like(x)
        check(lib().pt_apply_matvec(self._ctx, x.shape[0], _ptr(x), _ptr(y)), "pt_apply_matvec")
        return y

    def apply_R(self, x: torch.Tensor) -> torch.Tensor:
        y = torch.empty_like(x)
        check(lib().pt_apply_R(self._ctx, x.shape[0], _ptr(x), _ptr(y)), "pt_apply_R")
        return y

    def apply_D_inverse(self, x: torch.Tensor) -> torch.Tensor:
        y = torch.empty_like(x)
        check(lib().pt_apply_D_inverse(self._ctx, x.shape[0], _ptr(x), _ptr(y)), "pt_apply_D_inverse")
        return y

    def precond(self, x: torch.Tensor) -> torch.Tensor:
        y = torch.empty_like(x)
        check(lib().pt_apply_precond(self._ctx, x.shape[0], _ptr(x), _ptr(y), _ptr(self._scratch),
                                     self._scratch.numel()), "pt_apply_precond")
        return y

    def rhs(self, f: torch.Tensor) -> torch.Tensor:
        if f.dim() == 2:
            f = f.unsqueeze(0)
        S = self._check_src(f)
        y = self._vec(S)
        check(lib().pt_rhs(self._ctx, S, _ptr(f), _ptr(y), _ptr(self._scratch), self._scratch.numel()), "pt_rhs")
        return y

    def block(self, layer: int, j: int, k: int) -> torch.Tensor:
        """G^l(z_j, z_k) / h as an (n_t, n_t) complex128 CUDA tensor."""
        out = torch.empty((self.nt, self.nt), dtype=torch.complex128, device=self.device)
        check(lib().pt_get_block(self._ctx, layer, j, k, _ptr(out)), "pt_get_block")
        return out
