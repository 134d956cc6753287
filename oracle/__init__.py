"""CPU FP64 oracle for the partitioned shift-without-invert eigensolution.

TEST INFRASTRUCTURE ONLY.  Nothing in the library (``paper_1606_01139_gb300``)
imports, calls or links anything here; only ``tests/``, the smoke check in
``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` use it.

The oracle is plain, slow and written to be checked by eye against the paper
(Feldman & Zhou, "A partitioned shift-without-invert algorithm to improve
parallel eigensolution efficiency in real-space electronic transport"):

* ``stencil``   -- the operator A = H_KS - i Gamma of Eq. (1): 12th-order
                   finite-difference kinetic term, potential, absorbers; a
                   ghost-padded matvec and a dense Kronecker-sum matrix.
* ``eigen``     -- dense spectra (LAPACK zgeev through numpy), the U^T U = I
                   normalisation, and the paper's own per-window solver: ARPACK
                   'SM' on the shifted, never-inverted operator of Eq. (3).
* ``partition`` -- Algorithm 1 (window counts, shifts, hole-filling window),
                   Algorithm 2 (combine, de-duplicate, hole flags), the planner's
                   sample merge, and the window a complex shift delivers (the
                   two-dimensional partition of Section 2).
* ``refine``    -- the FP64 residual-correction sweep (Rayleigh-Ritz on
                   span[U, R] with the unconjugated pencil).
* ``transport`` -- T(E) = Tr{G Gamma_R G^dagger Gamma_L} (Section 1) from the
                   spectral G and from a dense inverse; the adjoint gradient
                   dT/dV(r), dT/dE, and central finite differences.

Every function is pinned by a ``-m "not gpu"`` test in ``tests/test_oracle_*``
against closed forms, invariants, brute force or values fixed by the paper.
No function here is "parity unpinned".
"""
