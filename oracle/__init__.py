"""CPU FP64 oracle for the coated half-space FFT-BEM (test infrastructure only).

This package is the slow, plainly written reference that the CUDA path is checked
against.  It is *test infrastructure*: only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it.  The product path (the
``paper_1807_01885_gb300`` package and its CUDA library) never imports, links or
calls anything here, and nothing here imports the product package: inputs come in
as plain numpy arrays.

Modules
-------
kernel    Fourier-space compliance of a layer bonded to a half-space (Eqs. 4, 9, 10),
          the rigid-base factor Lambda (Eq. 25), the DC finite part, and an
          independent plane-strain transfer-matrix solve of Eq. (5) with
          boundary conditions (a)-(d) used only to pin Eq. (9).
dft       naive O(M^2) DFT and a textbook iterative radix-2 FFT (no library FFT).
operator  the discrete operator u = K p of Eq. (1)/(11): wave-number grid, the
          dense influence matrix from a naive inverse DFT, and the FFT form.
contact   Polonsky-Keer constrained conjugate gradients (the method the paper
          cites for the inverse problem, Sec. 2), the KKT check, and the
          adhesive pull-off procedure with the detachment criterion of Eq. (12).
analytic  closed forms used as pins: Hertz, JKR, flat punch (Eq. 4 based),
          thin-layer Eqs. (13)-(21), thick-layer series Eqs. (22)-(25).
fno       FP64 Fourier-neural-operator forward/backward (naive truncated DFT),
          the reference for the warm-start network's kernels.
influence the non-periodic operator of a homogeneous half-space: Love's closed-form
          displacement of a uniformly loaded square cell, convolved over the open
          plane (no k = 0 convention); no CUDA counterpart yet.

Parity status: every function here is pinned by ``tests/test_oracle_*.py`` against
closed forms, limits, invariants, brute force or an independent derivation; see
each module's header.
"""
