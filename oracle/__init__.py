"""CPU oracle for the method of polarized traces (Zepeda-Nunez & Demanet, 2014).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, FP64 NumPy/SciPy
restatement of what the paper computes.  It exists so that the CUDA library
can be checked against something written independently of it.  Only the test
suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import it; the library and its Python binding never do, and this package
imports nothing from them.

Modules
-------
discretization  Section 2.1 (5-point Helmholtz with PML) and Section 2.2
                (layered decomposition, padded local problems).
green           Section 2.3: Definition 1 (interface Green's matrices),
                Definition 2 (incomplete Green's integrals), Definition 3
                (Newton potential), Lemma 1 (discrete GRF).
integral        Section 2.4: Definition 4 / Theorem 1 (unpolarized integral
                system) and Remark 1 (the M_0 system).
polarized       Section 3: Definitions 5, 6, 9, Lemmas 3-4, the four
                jump-condition equations, the permutation P and the splitting
                D + R; Section 4.1 Algorithms 3 and 4.
krylov          Section 4.2: GMRES (left preconditioned) and flexible GMRES
                (right preconditioned), Arnoldi with modified Gram-Schmidt and
                Givens rotations.
solver          Algorithm 2 end to end with the polarized system.
plr             Section 5.1: Algorithms 5 and 6 and the flattened leaf form.
learned         Not in the paper: the learned correction N_theta of the
                preconditioner used inside flexible GMRES (Section 4.2) -
                forward pass, loss, exact gradient, trace/feature maps and
                the defect targets e - K^{-1} r of Algorithm 4.

Parity status: every function here is pinned by a test in
``tests/test_oracle_*.py`` against an identity the paper proves, a closed
form, a library routine on a special case, or brute force on tiny inputs.
"""
