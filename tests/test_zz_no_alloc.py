"""pt_rhs_noalloc, the entry point for callers that cannot allocate device memory.

Some callers own no allocator: their device memory belongs to a host
framework's pool, or their serving loop must not call cudaMalloc after
start-up (the call can synchronise the device).  pt_rhs_noalloc gives them
the interface right-hand side of pt_rhs with its local-solve scratch in a
fixed 16 MiB array inside the library.  These tests call it through the C ABI
and compare with pt_rhs (caller-provided scratch) on two calls in a row with
different sources, so that contents left behind by the first call cannot
leak into the second.  This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu


def _solver(wl, max_sources):
    from paper_1410_5910_gb300 import PolarTrace

    c = wl.c_ext()
    return PolarTrace(wl.nx, wl.nz, wl.npml, wl.L, wl.h, wl.omega(c), torch.from_numpy(c).cuda(),
                      max_sources=max_sources)


def test_noalloc_rhs_equals_pt_rhs_on_two_calls_in_a_row():
    from paper_1410_5910_gb300._lib import lib

    wl = W.small_case(40, 60, 8, 3, medium="grf", seed=11)
    solver = _solver(wl, max_sources=2)
    inputs = [W.random_sources(wl.nt, wl.Nz, wl.npml, wl.nx, wl.nz, seed=21, count=2),
              W.point_sources(wl.nt, wl.Nz, wl.npml, wl.h, [(3, 4), (30, 50)])]
    for f_np in inputs:
        f = torch.from_numpy(f_np).cuda()
        ref = solver.rhs(f)  # pt_rhs with the caller's scratch
        y = torch.full_like(ref, complex(np.nan, np.nan))
        st = lib().pt_rhs_noalloc(solver._ctx, f.shape[0], f.data_ptr(), y.data_ptr())
        assert st == 0, lib().pt_last_error()
        torch.cuda.synchronize()
        err = float(torch.linalg.vector_norm(y - ref) / torch.linalg.vector_norm(ref))
        assert err <= 1e-12


def test_noalloc_rhs_rejects_requests_beyond_its_scratch():
    from paper_1410_5910_gb300._lib import lib

    wl = W.small_case(200, 300, 10, 4)
    solver = _solver(wl, max_sources=1)
    nsrc = 16  # 16 * 4 layers * 220 columns * 105 rows * 16 B > 16 MiB
    f = torch.zeros((nsrc, wl.Nz, wl.nt), dtype=torch.complex128, device="cuda")
    y = torch.zeros((nsrc, solver.T4, wl.nt), dtype=torch.complex128, device="cuda")
    st = lib().pt_rhs_noalloc(solver._ctx, nsrc, f.data_ptr(), y.data_ptr())
    assert st == 2  # PT_ERR_WORKSPACE
    assert b"16 MiB" in lib().pt_last_error()
