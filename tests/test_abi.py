"""The C-ABI library loads and exports every symbol include/polartrace.h declares (CPU only).

Also checks the host-only entry points (partition, workspace sizes, argument
validation) that need no GPU.
"""
import ctypes as C
import os
import re

import numpy as np
import pytest

from oracle import discretization as D

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "polartrace.h")


@pytest.fixture(scope="module")
def L():
    from paper_1410_5910_gb300 import _lib
    from paper_1410_5910_gb300.build import LIB, build

    if not os.path.exists(LIB):
        build()
    return _lib.lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pt_[A-Za-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n
    from paper_1410_5910_gb300 import _lib

    assert sorted(_lib.EXPORTS) == names


def test_symbols_in_shared_object_are_c_linkage():
    from paper_1410_5910_gb300.build import LIB

    if not os.path.exists(LIB):
        pytest.skip("library not built")
    import subprocess

    out = subprocess.run(["nm", "-D", "--defined-only", LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (pt_\w+)$", out, flags=re.M))
    assert set(declared_functions()) <= exported


def _params(L_, **kw):
    from paper_1410_5910_gb300._lib import Params

    d = dict(nx=128, nz=128, npml=10, L=4, h=1 / 129, omega=81.0, pml_C=20.0, precision=0, gs_iters=2,
             max_sources=1, max_krylov=30, plr=0, plr_eps=1e-9, plr_rmax=24)
    d.update(kw)
    return Params(**d)


@pytest.mark.parametrize("nz,npml,L_", [(128, 10, 4), (1023, 20, 16), (2047, 20, 32), (100, 7, 3)])
def test_partition_matches_oracle(L, nz, npml, L_):
    p = _params(L, nz=nz, npml=npml, L=L_)
    out = (C.c_int32 * (L_ + 1))()
    assert L.pt_layer_partition(C.byref(p), out) == 0
    assert list(out) == list(D.layer_partition(nz + 2 * npml, L_))


def test_workspace_sizes_and_validation(L):
    p = _params(L)
    a, b, c = C.c_size_t(), C.c_size_t(), C.c_size_t()
    assert L.pt_workspace_size(C.byref(p), C.byref(a), C.byref(b), C.byref(c)) == 0
    nt, L_ = 148, 4
    # at least the Green's blocks in FP64 and the local factors
    assert a.value >= L_ * 16 * nt * nt * 16
    p2 = _params(L, precision=1)
    a2 = C.c_size_t()
    assert L.pt_workspace_size(C.byref(p2), C.byref(a2), None, None) == 0
    assert a2.value > a.value  # FP32 copies of the blocks
    for bad in (dict(L=1), dict(h=0.0), dict(omega=-1.0), dict(gs_iters=0), dict(L=70), dict(npml=0),
                dict(precision=7), dict(max_krylov=0), dict(plr=1, plr_rmax=0), dict(plr=1, plr_rmax=40),
                dict(plr=1, plr_eps=0.0)):
        assert L.pt_workspace_size(C.byref(_params(L, **bad)), None, None, None) == 1, bad
    assert b"" != L.pt_last_error()
    assert L.pt_status_string(5) == b"GMRES did not converge"


def test_create_rejects_null_and_small_workspace_without_touching_the_gpu(L):
    p = _params(L)
    ctx = C.c_void_p()
    assert L.pt_create(C.byref(p), None, None, 0, None, 0, None, C.byref(ctx)) == 1
    assert L.pt_create(C.byref(p), C.c_void_p(256), C.c_void_p(256), 16, C.c_void_p(512), 16, None,
                       C.byref(ctx)) == 2
    assert not ctx.value


def test_mixed_form_workspace_holds_its_copies_and_chunk_transfer_matrices(L):
    """Host-side sizes of the mixed FP32 form: the persistent workspace grows by at least the complex64 hi / lo
    and FP16 block copies and the chunk transfer matrices (K_r + K_v chunks per layer, three n x n complex64
    matrices each); the setup workspace holds the FP64 scratch the transfer matrices are formed in."""
    nx, nz, npml, L_ = 128, 128, 10, 4
    nt = nx + 2 * npml
    ld32 = (nt + 3) & ~3
    starts = D.layer_partition(nz + 2 * npml, L_)
    nloc = [int(starts[l + 1] - starts[l]) + (npml if l > 0 else 0) + (npml if l < L_ - 1 else 0) for l in range(L_)]
    nmax = max(nloc)
    kmax = max(1, min(64, nt // 16))
    kr = min(kmax, 32)
    a64, a32, s32 = C.c_size_t(), C.c_size_t(), C.c_size_t()
    assert L.pt_workspace_size(C.byref(_params(L, precision=0)), C.byref(a64), None, None) == 0
    assert L.pt_workspace_size(C.byref(_params(L, precision=1)), C.byref(a32), C.byref(s32), None) == 0
    copies = L_ * 16 * nt * ld32 * (8 + 8 + 4)
    # K_v is at least 1 and at most kmax (it depends on the SM count of the device, if there is one)
    transfer_min = L_ * (kr + 1) * 3 * nmax * nmax * 8
    assert a32.value - a64.value >= copies + transfer_min
    assert s32.value >= L_ * kr * 4 * nmax * nmax * 16
    # options are per context: a NULL context is an argument error, not a crash
    assert L.pt_set_option(None, 6, 1) == 1


def test_layer_rows_set_the_partition_and_are_validated(L):
    """Section 2.2 allows any increasing sequence of interfaces: pt_params.layer_rows gives the rows per
    layer; the library must use exactly that split and reject sums other than N_z, layers under 3 rows
    and interfaces in or next to the PML, before touching the GPU."""
    nz, npml, L_ = 128, 10, 4
    Nz = nz + 2 * npml
    rows = [50, 22, 41, Nz - 113]
    arr = (C.c_int32 * L_)(*rows)
    p = _params(L, nz=nz, npml=npml, L=L_, layer_rows=C.cast(arr, C.POINTER(C.c_int32)))
    out = (C.c_int32 * (L_ + 1))()
    assert L.pt_layer_partition(C.byref(p), out) == 0
    assert list(out) == [0, 50, 72, 113, Nz]
    assert L.pt_workspace_size(C.byref(p), None, None, None) == 0
    for bad in ([50, 22, 41, Nz - 112],      # sum N_z + 1
                [50, 2, 61, Nz - 113],       # a layer of 2 rows
                [10, 62, 41, Nz - 113],      # first interface at row 10 = inside the 10-row PML
                [50, 22, Nz - 82, 10]):      # last interface at row 138 > N_z - npml - 1 = 137
        arr_b = (C.c_int32 * L_)(*bad)
        pb = _params(L, nz=nz, npml=npml, L=L_, layer_rows=C.cast(arr_b, C.POINTER(C.c_int32)))
        assert L.pt_layer_partition(C.byref(pb), out) == 1, bad
