"""Plain FP64 CPU oracle for MGRIT/Parareal on periodic linear advection.

TEST INFRASTRUCTURE ONLY.  This package restates the method of De Sterck,
Falgout, Friedhoff, Krzysik and MacLachlan, "Optimizing MGRIT and Parareal
coarse-grid operators for linear advection" (Numer. Linear Algebra Appl.,
2021), in slow, obviously correct numpy: full space-time storage, stage-by-
stage Runge-Kutta, circulant solves by FFT division, and LAPACK least squares.
It shares no code with the CUDA library in ``paper_1910_03726_gb300`` and
neither package imports the other.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py`` (its ``cpu_baseline`` leg and its
``--impl reference`` arm) may import it; the product path never does.

Modules
-------
schemes   U1..U5 stencils (Section 2.1), ERK/SDIRK tableaux (Appendix A),
          stability function and Fourier symbol (Lemma 1), CFL limits (Table 1).
stepping  the fine propagator Phi (Eq. 3) and sequential time stepping.
psi       first column of Phi^m, sparsity patterns (Section 4.2, 4.3, 4.6),
          the weighted least-squares fit (Eq. 6), the two-level bound (Eq. 4)
          and operator complexity (Eq. 5).
mgrit     two-level and multilevel FCF-MGRIT with full storage (Section 2.2).

Parity pins: every function is checked in ``tests/test_oracle_*.py`` against
values the paper prints, closed forms, or invariants of the method; see the
header of each module for the list.
"""
