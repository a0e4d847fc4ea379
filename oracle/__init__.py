"""FP64 CPU oracle for the symmetric stair preconditioned CG path.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package; the library in
``paper_2309_06427_gb300`` never does, and this package never imports it.

Two independent routes to the same result:

* ``oracle.block`` (C, ``sspcg_oracle.c``): the paper's block formulas
  (Sec. II-A), stair inverses (Eq. stair_inv), the symmetric/additive stair
  combinations (Sec. III, Sec. IV) and textbook PCG, in FP64.
* ``oracle.dense`` (numpy/scipy): the definitions written out densely,
  S = C G^-1 C^T from the KKT matrices, Psi_l/Psi_r/P_l/P_r by their block
  patterns, inverses by LAPACK, a dense Cholesky solve and dense spectra.
"""
